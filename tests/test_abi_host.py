"""C-ABI library: loads, exports every declared symbol, and validates its
arguments on the host before touching the GPU (CPU only, no compute)."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

import mdgen
from paper_1408_4599_gb300 import md

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(md_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_builds_and_loads():
    import __graft_entry__ as g
    g.build()
    assert os.path.exists(md.LIB_PATH)
    md.lib()


def test_exports_every_declared_symbol():
    L = md.lib()
    declared = _declared_functions()
    assert len(declared) >= 14
    missing = [n for n in declared if not hasattr(L, n)]
    assert missing == []
    assert set(md.EXPORTS) <= set(declared)


def test_status_strings():
    L = md.lib()
    for code in md.STATUS:
        assert L.md_status_str(code).decode().startswith(md.STATUS[code])


def _create(box=(10.0, 10.0, 10.0), rc=2.5, model=None, **kw):
    return md.md_create(box, rc, model or mdgen.model_lj(), **kw)


def test_box_smaller_than_two_cutoffs_is_rejected():
    with pytest.raises(md.MDError) as e:
        _create(box=(10.0, 4.9, 10.0), rc=2.5)
    assert e.value.code == -2


@pytest.mark.parametrize("bad", [
    dict(rc=-1.0), dict(rc=float("nan")), dict(box=(10.0, float("inf"), 10.0)),
    dict(eps_rf=0.5), dict(eps_rf=float("nan")), dict(cell_div=3), dict(cell_div=-1),
])
def test_bad_scalars_are_rejected(bad):
    with pytest.raises(md.MDError) as e:
        _create(**bad)
    assert e.value.code == -1


def test_bad_models_are_rejected():
    m = mdgen.model_lj()
    m["lj"][0]["type"] = 3
    with pytest.raises(md.MDError) as e:
        _create(model=m)
    assert e.value.code == -1
    m = mdgen.model_2cljq()
    m["lj"][0]["pos"] = (0.0, 0.0, -0.3)  # centre of mass off the origin
    with pytest.raises(md.MDError) as e:
        _create(model=m)
    assert e.value.code == -1
    m = mdgen.model_lj()
    m["lj_types"]["sigma"] = [0.0]
    with pytest.raises(md.MDError) as e:
        _create(model=m)
    assert e.value.code == -1
    m = mdgen.model_lj()
    m["lj"] = [{"pos": (0.1 * k, 0.0, 0.0), "type": 0, "mass": 0.0} for k in range(9)]
    with pytest.raises(md.MDError) as e:
        _create(model=m)
    assert e.value.code == -9  # more merged sites than supported


def test_batch_rejects_half_cutoff_cells():
    """Replicas use cells of edge >= cutoff: cell_div = 2 is refused before
    anything is allocated."""
    M = md.Model(mdgen.model_lj())
    boxes = (C.c_double * 6)(10.0, 10.0, 10.0, 12.0, 12.0, 12.0)
    h = C.c_void_p()
    for div, code in ((2, -9), (3, -1)):
        o = md.md_options(math.inf, 0, 0, 0, 1, div)
        assert md.lib().md_batch_create(2, boxes, 2.5, C.byref(M.types), C.byref(o), C.byref(h)) == code
        assert not h.value


def test_null_handle_calls_fail_cleanly():
    L = md.lib()
    assert L.md_compute_forces(None, None) == -1
    assert L.md_step(None, 1, 0.001, 0.0, None) == -1
    assert L.md_energy_virial(None, None) == -1
    assert L.md_n_molecules(None) == -1
    L.md_destroy(None)


def test_binding_refuses_mismatched_state_shapes():
    """The library reads n rows of every state array (n from r), so the
    binding refuses arrays of other shapes before any library call."""
    r = np.zeros((5, 3))
    with pytest.raises(ValueError, match=r"q has shape \(4, 4\)"):
        md.md_set_molecules(None, r, np.zeros((4, 4)))
    with pytest.raises(ValueError, match=r"v has shape \(5, 4\)"):
        md.md_set_molecules(None, r, np.zeros((5, 4)), v=np.zeros((5, 4)))
    with pytest.raises(ValueError, match=r"r has shape \(15,\)"):
        md.md_set_molecules(None, r.ravel(), np.zeros((5, 4)))


def test_binding_refuses_outputs_it_would_have_to_copy():
    """Host output arrays are written through their pointer: a float32,
    strided or read-only array would receive nothing, so it is refused."""
    for bad in (np.zeros((4, 3), dtype=np.float32), np.zeros((4, 6))[:, ::2]):
        with pytest.raises(ValueError, match="writable C-contiguous float64"):
            md.md_get_forces(None, F=bad)
        with pytest.raises(ValueError, match="writable C-contiguous float64"):
            md.md_get_molecules(None, r=bad)
    ro = np.zeros((4, 3))
    ro.flags.writeable = False
    with pytest.raises(ValueError, match="writable C-contiguous float64"):
        md.md_get_molecules(None, v=ro)
    # inputs of another dtype or layout are converted, not refused
    p, on_dev, keep = md._ptr(np.zeros((4, 6), dtype=np.float32)[:, ::2])
    assert on_dev == 0 and keep.dtype == np.float64 and keep.flags["C_CONTIGUOUS"]


def test_binding_refuses_misshaped_ensembles():
    with pytest.raises(ValueError, match="n_cfg x n x 3"):
        md.md_param_grad(None, np.zeros((2, 5, 3)), np.zeros((2, 4, 4)))
    with pytest.raises(ValueError, match="n_cfg x n x 3"):
        md.md_param_grad(None, np.zeros((5, 3)), np.zeros((5, 4)))


class _FakeCudaTensor:
    """Stands in for a CUDA tensor on a CPU-only machine: the binding sees
    on_device = 1 for it (through a patched _ptr) and never dereferences it."""

    def __init__(self, shape, index=0):
        self.shape = shape
        self.device = type("Dev", (), {"index": index, "__str__": lambda s: f"cuda:{index}"})()


def _patch_fake_cuda(monkeypatch):
    real = md._ptr

    def fake_ptr(a, out=False):
        if isinstance(a, _FakeCudaTensor):
            return C.c_void_p(0x1000), 1, a
        return real(a, out)

    monkeypatch.setattr(md, "_ptr", fake_ptr)
    monkeypatch.setattr(md, "lib", lambda: pytest.fail("the library was called"))


def test_binding_refuses_host_outputs_mixed_with_device_outputs(monkeypatch):
    """md_get_molecules / md_get_forces take one on_device flag for all
    pointers: a host array beside a CUDA tensor would reach a kernel as a
    device address, so the mix is refused before any library call."""
    _patch_fake_cuda(monkeypatch)
    with pytest.raises(ValueError, match="same side"):
        md.md_get_molecules(None, r=np.zeros((4, 3)), v=_FakeCudaTensor((4, 3)))
    with pytest.raises(ValueError, match="same side"):
        md.md_get_forces(None, F=np.zeros((4, 3)), tau=_FakeCudaTensor((4, 3)))
    with pytest.raises(ValueError, match="same side"):
        md.md_set_molecules(None, np.zeros((4, 3)), _FakeCudaTensor((4, 4)))


def test_binding_refuses_tensors_off_the_current_device(monkeypatch):
    """The library launches on the current device, so a CUDA tensor on any
    other device is refused (md_kinetic_noalloc's scratch is per device)."""
    torch = pytest.importorskip("torch")
    _patch_fake_cuda(monkeypatch)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    with pytest.raises(ValueError, match="current device is cuda:0"):
        md.md_get_forces(None, F=_FakeCudaTensor((4, 3), 0), tau=_FakeCudaTensor((4, 3), 1))
    t3 = [_FakeCudaTensor((4, 3), 0) for _ in range(4)]
    with pytest.raises(ValueError, match="current device is cuda:0"):
        md.md_kinetic_noalloc(t3[0], _FakeCudaTensor((4, 4), 1), t3[1], t3[2], t3[3], 1.0, (1.0, 1.0, 0.0), 0.001,
                              _FakeCudaTensor((2,), 0))
