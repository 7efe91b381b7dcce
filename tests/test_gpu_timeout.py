"""A bounded device wait that runs out, made to happen without any fault: the
G_x offset scan's look-back waits for the words its predecessor tiles publish.
The test hook keeps one tile from publishing and lowers the wait bound, so the
later tiles' waits run out.  They flag the error, take their prefix from a
direct sum instead, and rs_score returns RS_ETIMEOUT; the scores stay exact."""
import numpy as np
import pytest

import graphgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_01485_gb300 as rsgpu
    return rsgpu


@pytest.mark.parametrize("tile", [0, 1, 3])
def test_scan_wait_runs_out_and_reports_timeout(rs, tile):
    g = graphgen.dcsbm_small(20000, seed=3)           # 5 tiles of 4,096 nodes
    G = rs.Graph.from_generated(g)
    ref, wmax = G.score(want_omega_max=True)
    ref = ref.cpu().numpy()
    assert G.device_errors() == 0
    G.test_gx_stall(tile, spin_limit=1000)
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    with pytest.raises(rs.RSError) as ex:
        G.score(out=out, want_omega_max=True)
    assert ex.value.status == rs.RS_ETIMEOUT
    assert G.device_errors() & 32
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    # back to the normal scan: no error, the same bits
    G.test_gx_stall(-1)
    again, w2 = G.score(want_omega_max=True)
    assert G.device_errors() == 0 and w2 == wmax
    np.testing.assert_array_equal(again.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    G.close()


def test_last_tile_withheld_is_harmless(rs):
    """No tile waits for the last one: nothing runs out."""
    g = graphgen.dcsbm_small(20000, seed=3)
    G = rs.Graph.from_generated(g)
    ref = G.score().cpu().numpy()
    G.test_gx_stall(4, spin_limit=1000)
    got, _ = G.score(want_omega_max=True)
    assert G.device_errors() == 0
    np.testing.assert_array_equal(got.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    G.close()
