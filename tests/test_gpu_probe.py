"""The roofline microbenchmarks run and report physically possible numbers:
conflict-free shared loads at most the nominal 128 bytes per clock per SM
(and most of it), scattered interval loads and atomics below that, and an L2
read bandwidth above the HBM copy bandwidth of the part."""
import pytest

import paper_2207_12116_gb300 as pccp
from paper_2207_12116_gb300 import _abi

pytestmark = pytest.mark.gpu


def test_probe_rejects_unknown_kind():
    with pytest.raises(pccp.PccpError) as e:
        pccp.pccp_probe(7)
    assert e.value.code == pccp.PCCP_ERR_INVALID


def test_probes_are_physical():
    p = pccp.roofline_probes()
    load = p["smem_load"]["per_clk_per_sm"]
    assert 64 <= load <= 128 * 1.02, p
    assert 0 < p["smem_scattered_v2"]["per_clk_per_sm"] <= load * 1.02, p
    assert 0 < p["smem_atomic"]["per_clk_per_sm"] <= 32 * 1.02, p  # one warp-wide op per clock
    assert 4000 < p["l2_read"]["gbs"] < 60000, p
    for v in p.values():
        assert 500 < v["sm_mhz"] < 2200, p


def test_probe_work_counts_scale_with_iterations():
    a = pccp.pccp_probe(_abi.PCCP_PROBE_SMEM_LOAD, 2000)
    b = pccp.pccp_probe(_abi.PCCP_PROBE_SMEM_LOAD, 4000)
    assert b["work"] == 2 * a["work"]
    assert b["ms"] > 1.3 * a["ms"]
