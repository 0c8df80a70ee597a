"""The H^2-compressed scattering apply (rte_h2_*, Section 5.2) against the
oracle's H^2 approximation.

* the block tree the library builds has the oracle's far and near blocks;
* Y = X S^+ and Y = X S^- element by element against the oracle's
  approximated matrix: FP64 to 1e-12, FP32 to 2e-5, BF16 on the tensor
  cores to 4 unit roundoffs of BF16 relative to max|Y| (about ten BF16
  roundings lie in sequence along the far-field path, mostly independent:
  measured 1.3 to 1.43 units), at
  n_S^+ = 1024 (far blocks at the leaf depth only) and n_S^+ = 4096 (far
  blocks on two depths: the transfer matrices), ragged row counts;
* n_S^+ = 256 has no admissible block: the apply is the dense matrix;
* the compression error against the library's own dense matrix at the
  paper's parameters stays within the oracle-pinned 3e-4;
* refusals: unbuilt parity or precision, misaligned arrays.
"""
import numpy as np
import pytest

from oracle import h2 as oh2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')

G = 0.5
_ORACLE = {}


def oracle_matrix(levels, parity):
    key = (levels, parity)
    if key not in _ORACLE:
        H = _ORACLE.setdefault(('H', levels), oh2.H2Scattering(levels, G))
        _ORACLE[key] = H.approximate(parity)
    return _ORACLE[key]


@pytest.fixture(scope='module')
def h2lib():
    import paper_2102_09038_gb300 as rte
    made = {}

    def get(levels, **kw):
        key = (levels, tuple(sorted(kw.items())))
        if key not in made:
            made[key] = rte.H2Scattering(levels, G, **kw)
        return made[key]
    yield get
    for h in made.values():
        h.close()


@pytest.mark.parametrize('levels', [4, 5])
def test_block_tree_matches_oracle(h2lib, levels):
    H = oh2.H2Scattering(levels, G)
    info = h2lib(levels).info()
    far = tuple(sum(1 for b in H.far if b[3] == s) for s in (1.0, -1.0))
    near = tuple(sum(1 for b in H.near if b[3] == s) for s in (1.0, -1.0))
    assert info['far_blocks'] == far and info['near_blocks'] == near
    assert info['leaves'] == 4 * 4 ** (levels - 3)
    assert info['n_plus'] == 4 * 4 ** levels


@pytest.mark.parametrize('levels, parity, rows', [(4, 1, 130), (4, -1, 63), (5, 1, 65)])
def test_apply_matches_oracle(h2lib, levels, parity, rows):
    import paper_2102_09038_gb300 as rte
    S = oracle_matrix(levels, parity)
    n = S.shape[0]
    X = np.random.default_rng(levels * 10 + rows).standard_normal((rows, n))
    ref = X @ S.T
    h = h2lib(levels)
    xt = torch.tensor(X, dtype=torch.float64, device='cuda')
    y64 = h.apply(xt, parity=parity, precision=rte.FP64).cpu().numpy()
    y32 = h.apply(xt, parity=parity, precision=rte.MIXED_FP32).cpu().numpy()
    ybf = h.apply(xt, parity=parity, precision=rte.MIXED_BF16).cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(y64 - ref).max() <= 1e-12 * scale
    assert np.abs(y32 - ref).max() <= 2e-5 * scale
    assert np.abs(ybf - ref).max() <= 4 * 2.0 ** -9 * scale


def test_no_admissible_block_is_dense(h2lib):
    import paper_2102_09038_gb300 as rte
    h = h2lib(3)
    info = h.info()
    assert info['far_blocks'] == (0, 0)
    for parity in (1, -1):
        D = h.dense(parity)
        X = np.random.default_rng(7).standard_normal((33, D.shape[0]))
        y = h.apply(torch.tensor(X, device='cuda'), parity=parity, precision=rte.FP64)
        ref = X @ D.T
        assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


def test_compression_error_against_dense(h2lib):
    import paper_2102_09038_gb300 as rte
    h = h2lib(5)
    for parity in (1, -1):
        D = h.dense(parity)
        X = np.random.default_rng(3).standard_normal((16, D.shape[0]))
        ref = X @ D.T
        y = h.apply(torch.tensor(X, device='cuda'), parity=parity,
                    precision=rte.FP64).cpu().numpy()
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 3e-4


def test_rows_zero_and_refusals(h2lib):
    import paper_2102_09038_gb300 as rte
    h = rte.H2Scattering(4, G, parities=1, precisions=1)
    try:
        x = torch.zeros((0, h.n_plus), dtype=torch.float64, device='cuda')
        assert h.apply(x).shape == (0, h.n_plus)
        x = torch.zeros((4, 3 * h.n_plus), dtype=torch.float64, device='cuda')
        with pytest.raises(rte.RteError, match='parity was not built'):
            h.apply(x, parity=-1)
        x = torch.zeros((4, h.n_plus), dtype=torch.float64, device='cuda')
        with pytest.raises(rte.RteError, match='precision was not built'):
            h.apply(x, precision=rte.MIXED_FP32)
        with pytest.raises(rte.RteError, match='precision was not built'):
            h.apply(x, precision=rte.MIXED_BF16)
        big = torch.zeros((4 * h.n_plus + 1,), dtype=torch.float64, device='cuda')
        xm = big[1:].view(4, h.n_plus)
        with pytest.raises(rte.RteError, match='16-byte aligned'):
            h.apply(xm)
    finally:
        h.close()
