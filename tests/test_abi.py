"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point include/pccp.h declares, and rejects malformed models on
the host before touching the GPU."""
import os
import re

import numpy as np
import pytest

import paper_2207_12116_gb300 as pccp
from paper_2207_12116_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header="pccp.h"):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pccp_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    lib = pccp.load()
    names = declared_functions()
    assert len(names) >= 8
    for n in names:
        assert hasattr(lib, n), n
        assert n in _abi.SIGNATURES, f"binding lacks {n}"


def test_binding_constants_match_the_headers():
    """Every integer #define of the headers has the same value in the binding."""
    seen = 0
    for header in ("pccp.h", "pccp_probe.h"):
        text = open(os.path.join(ROOT, "include", header)).read()
        for name, val in re.findall(r"^#define[ \t]+(PCCP_[A-Z0-9_]+)[ \t]+(.+?)[ \t]*(?:/\*.*)?$", text,
                                    flags=re.M):
            m = re.fullmatch(r"\(?(-?\d+)u?(?:\s*<<\s*(\d+))?\)?", val)
            assert m, (name, val)
            want = int(m.group(1)) << int(m.group(2) or 0)
            assert getattr(_abi, name) == want, name
            seen += 1
    assert seen >= 20


def test_probe_library_exports_every_declared_entry_point():
    lib = _abi.load_probe()
    names = declared_functions("pccp_probe.h")
    assert names == ["pccp_probe"]
    for n in names:
        assert hasattr(lib, n), n
        assert n in _abi.PROBE_SIGNATURES, f"binding lacks {n}"


def test_every_header_is_covered():
    assert sorted(os.listdir(os.path.join(ROOT, "include"))) == ["pccp.h", "pccp_probe.h"]


def test_error_strings():
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert pccp.pccp_error_string(code)
    assert pccp.pccp_error_string(-99) == "unknown error"


def _create(**kw):
    base = dict(lb0=[0, 0, 0], ub0=[5, 5, 1])
    base.update(kw)
    return pccp.Model(**base)


@pytest.mark.parametrize("kw, code", [
    (dict(lb0=[3, 0, 0], ub0=[2, 5, 1]), pccp.PCCP_ERR_INVALID),            # lb0 > ub0
    (dict(temporal=[[0, 7, 1]]), pccp.PCCP_ERR_INVALID),                     # index out of range
    (dict(reified=[[0, 1, 0, 2]]), pccp.PCCP_ERR_INVALID),                   # b not Boolean
    (dict(reified=[[2, 0, 1, 40000]]), pccp.PCCP_ERR_UNSUPPORTED),          # d beyond int16
    (dict(linear_c=[3], linear_off=[0, 1], term_coef=[0], term_var=[0]), pccp.PCCP_ERR_INVALID),
    (dict(linear_c=[3], linear_off=[0, 1], term_coef=[40000], term_var=[0]), pccp.PCCP_ERR_UNSUPPORTED),
    (dict(linear_c=[3], linear_off=[1, 1], term_coef=[1], term_var=[0]), pccp.PCCP_ERR_INVALID),
    (dict(lb0=[0, 0, 0], ub0=[1 << 30, 5, 1]), pccp.PCCP_ERR_OVERFLOW),     # value limit
    (dict(lb0=[0, 0, 0], ub0=[(1 << 29), 5, 1], linear_c=[0], linear_off=[0, 2],
          term_coef=[3, 1], term_var=[0, 1]), pccp.PCCP_ERR_OVERFLOW),      # sum could overflow
    (dict(objective=3), pccp.PCCP_ERR_INVALID),
    (dict(branch=[0, 9]), pccp.PCCP_ERR_INVALID),
])
def test_model_create_rejects_on_host(kw, code):
    with pytest.raises(pccp.PccpError) as e:
        _create(**kw)
    assert e.value.code == code


def test_many_variables_unsupported():
    with pytest.raises(pccp.PccpError) as e:
        pccp.Model(np.zeros(70000), np.ones(70000))
    assert e.value.code == pccp.PCCP_ERR_UNSUPPORTED
