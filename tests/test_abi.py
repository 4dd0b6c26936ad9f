"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point include/flamerec.h declares; the binding's
signatures cover exactly those declarations."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "flamerec.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(fr_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return set(names)


def test_library_exports_every_declared_symbol():
    from paper_1809_06417_gb300 import flamerec
    lib = flamerec.load()
    declared = _declared()
    assert {"fr_render", "fr_adjust", "fr_reconstruct", "fr_render_backward"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(flamerec.SIGNATURES) == declared


def test_abi_version_and_defaults():
    from paper_1809_06417_gb300 import flamerec
    lib = flamerec.load()
    assert lib.fr_abi_version() == 1
    p = flamerec.params()
    # the paper's constants (Sec. 4.1, 4.2, 5.1)
    assert p.step == 1.0 and abs(p.alpha_l - 0.001) < 1e-9 and p.alpha_d == 1.0
    assert abs(p.flame_thresh - 30 / 255) < 1e-7 and p.clamp_nonneg == 1


def test_struct_layouts():
    from paper_1809_06417_gb300 import flamerec
    assert ctypes.sizeof(flamerec.fr_camera) == 64
    assert ctypes.sizeof(flamerec.fr_volume) == 48
    assert flamerec.fr_params.lut.offset % 8 == 0


def test_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        return
    from paper_1809_06417_gb300 import flamerec
    lib = flamerec.load()
    h = ctypes.c_void_p()
    assert lib.fr_create(ctypes.byref(h), 0, None) == flamerec.FR_ECUDA
    assert not h.value


def test_host_only_entry_points_without_a_gpu():
    """The normal build has its bounds checks compiled out; the host-arithmetic
    entry points answer without a device."""
    from paper_1809_06417_gb300 import flamerec
    lib = flamerec.load()
    assert lib.fr_checks_enabled() == 0
    P = (ctypes.c_double * 12)(*([0.0] * 12))
    cam = flamerec.fr_camera()
    assert lib.fr_camera_from_projection(P, 8, 8, ctypes.byref(cam)) == flamerec.FR_EINVAL
