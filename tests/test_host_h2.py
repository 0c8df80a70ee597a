"""The host half of the H^2 compression (cluster tree, boxes, admissibility,
block tree) in the library against the oracle's, without a GPU: the far and
near block counts of both parts, the merged near matrices and the transfer
count, over sphere sizes where the block tree has one, two and three depths
of far blocks, and at another admissibility parameter and degree."""
import pytest

from oracle import h2 as oh2


@pytest.fixture(scope='module', autouse=True)
def lib_path():
    # the library is built here when it is missing (nvcc cross-compiles
    # without a GPU); the plan needs no device
    from paper_2102_09038_gb300 import build
    return build.build()


def oracle_counts(levels, eta, p):
    H = oh2.H2Scattering(levels, 0.5, eta=eta, p=p)
    far = tuple(sum(1 for b in H.far if b[3] == s) for s in (1.0, -1.0))
    near = tuple(sum(1 for b in H.near if b[3] == s) for s in (1.0, -1.0))
    merged = len({(b[1], b[2]) for b in H.near})
    dmin = min([b[0] for b in H.far] + [H.tree.leaf_depth])
    clusters = sum(H.tree.count(d) for d in range(dmin, H.tree.leaf_depth + 1))
    return far, near, merged, clusters - H.tree.count(dmin)


@pytest.mark.parametrize('levels, eta, p', [(3, 1.4, 4), (4, 1.4, 4), (5, 1.4, 4), (6, 1.4, 4),
                                            (5, 0.8, 3)])
def test_block_tree_counts_match_oracle(levels, eta, p):
    import paper_2102_09038_gb300 as rte
    got = rte.h2_plan_info(levels, eta=eta, p=p)
    far, near, merged, transfers = oracle_counts(levels, eta, p)
    assert got['far_blocks'] == far and got['near_blocks'] == near
    assert got['near_matrices'] == merged
    assert got['transfers'] == transfers
    assert got['n_plus'] == 4 * 4 ** levels and got['leaves'] == 4 * 4 ** (levels - 3)


def test_plan_refuses_bad_options():
    import paper_2102_09038_gb300 as rte
    with pytest.raises(rte.RteError, match='levels'):
        rte.h2_plan_info(2)
    with pytest.raises(rte.RteError, match='eta'):
        rte.h2_plan_info(4, eta=0.0)
    with pytest.raises(rte.RteError, match='p must'):
        rte.h2_plan_info(4, p=5)
