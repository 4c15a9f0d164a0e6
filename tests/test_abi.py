"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads
without a GPU, and exports every entry point that include/maxent.h declares;
the Python binding carries the same names.  No compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
            if f.endswith(".h")]
    names = set()
    for h in hdrs:
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(mxe_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for must in ["mxe_create", "mxe_destroy", "mxe_set_state", "mxe_set_bc",
                 "mxe_set_relaxation", "mxe_step", "mxe_get_moments", "mxe_get_diagnostics",
                 "mxe_last_error", "mxe_batch_create", "mxe_batch_run"]:
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    import paper_2401_15233_gb300 as mx
    L = mx.lib()
    for name in declared_entry_points():
        assert hasattr(L, name), name
        assert hasattr(mx, name), f"binding lacks {name}"


def test_config_struct_matches_header_field_order():
    import paper_2401_15233_gb300 as mx
    txt = open(os.path.join(ROOT, "include", "maxent.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} mxe_config;", txt, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"([a-z_0-9]+)\s*[,;]", body)
    assert fields == [f for f, _ in mx.Config._fields_]
    rest = txt.split("} mxe_config;")[1]
    body = re.search(r"typedef struct \{(.*?)\} mxe_diag;", rest, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"([a-z_0-9]+)(?:\[\d+\])?\s*;", body)
    assert fields == [f for f, _ in mx.Diag._fields_]


def test_invalid_config_rejected_without_gpu():
    """Validation happens before any device call."""
    import paper_2401_15233_gb300 as mx
    for bad in [dict(system=7), dict(system=5, ny=8), dict(cfl=0.0), dict(order=3),
                dict(sigma_lim=0.0), dict(k_ws=0.5), dict(nx=2), dict(nx=0), dict(ny=0),
                dict(nx=-5), dict(nx=3, ny=3)]:
        with pytest.raises(mx.MaxentError) as e:
            mx.Solver(**bad)
        assert e.value.status == mx.EINVAL


def test_invalid_batches_rejected_without_gpu():
    """Empty batches, empty or too short tubes, non-positive lengths and the
    5-moment mixed batch (mixed precision is 14-moment only)."""
    import paper_2401_15233_gb300 as mx
    for ncells, lengths, kw in [([], [], {}), ([0], [1.0], {}), ([100, 2], [1.0, 1.0], {}),
                                ([100], [0.0], {}), ([100], [-1.0], {}), ([100], [], {}),
                                ([100], [1.0], dict(system=5, precision="mixed"))]:
        with pytest.raises(mx.MaxentError) as e:
            mx.Batch(ncells, lengths, **({"system": 14} | kw))
        assert e.value.status == mx.EINVAL, (ncells, lengths, kw)


def test_binding_checks_array_size_before_passing_a_pointer():
    """The library trusts its pointers; the binding refuses an array whose
    element count differs from what the call will read or write."""
    import numpy as np
    import paper_2401_15233_gb300 as mx
    p, dev = mx._ptr(np.zeros(6), 6)
    assert dev == 0 and p.value is not None
    with pytest.raises(ValueError):
        mx._ptr(np.zeros(5), 6)
    with pytest.raises(ValueError):
        mx._ptr(np.zeros(6, dtype=np.float32), 6)
    with pytest.raises(ValueError):
        mx._state_elems(mx._P(12345))      # not a live context
