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
    assert lib.fr_abi_version() == 3
    p = flamerec.params()
    # the paper's constants (Sec. 4.1, 4.2, 5.1)
    assert p.step == 1.0 and abs(p.alpha_l - 0.001) < 1e-9 and p.alpha_d == 1.0
    assert abs(p.flame_thresh - 30 / 255) < 1e-7 and p.clamp_nonneg == 1


def test_struct_layouts():
    """The binding's structures have the header's sizes and field offsets (a C
    program compiled against include/flamerec.h prints them)."""
    import subprocess
    import tempfile
    from paper_1809_06417_gb300 import flamerec as fr
    assert ctypes.sizeof(fr.fr_camera) == 64
    assert ctypes.sizeof(fr.fr_volume) == 48
    assert fr.fr_params.lut.offset % 8 == 0
    fields = {"fr_params": ["lut", "hull_tags", "hg_g", "sequential_views", "tables"],
              "fr_problem": ["targets", "rmse", "hull_tags"],
              "fr_job_desc": ["cams", "init_records", "rmse", "hull_tags"],
              "fr_job_info": ["t_submit", "footprint"]}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "flamerec.h"', "int main(void) {"]
    for st, names in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in names:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines += ["return 0; }"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    got = dict(zip(out[0::2], (int(x) for x in out[1::2])))
    for st, names in fields.items():
        cls = getattr(fr, st)
        assert ctypes.sizeof(cls) == got[st], st
        for f in names:
            assert getattr(cls, f).offset == got[f"{st}.{f}"], (st, f)


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
