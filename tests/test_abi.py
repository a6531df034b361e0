"""CPU checks of the boundary: the library builds, loads and exports every
function that include/gc4d.h declares; the binding's ctypes layouts match the
header's structs.  No compute call is made (there may be no GPU here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gc4d.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^GC_API\s+[^;(]*?\b(gc_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def built():
    from paper_2509_17513_b300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gc_create", "gc_destroy", "gc_render_forward", "gc_render_backward",
                 "gc_saved_create", "gc_saved_destroy", "gc_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.check_output(["nm", "-D", "--defined-only", built], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_declares_every_symbol(built):
    from paper_2509_17513_b300 import _abi
    assert sorted(_abi.SIGNATURES) == _declared()
    L = C.CDLL(built)
    for n in _declared():
        assert hasattr(L, n)


def test_version_and_default_options_without_gpu(built):
    from paper_2509_17513_b300 import _abi
    L = _abi.lib()
    assert L.gc_version().startswith(b"gc4d")
    o = _abi.Options()
    assert L.gc_default_options(C.byref(o)) == 0
    assert (o.tile_w, o.tile_h) == (16, 16)
    assert abs(o.near_plane - 0.2) < 1e-7 and abs(o.dilation - 0.3) < 1e-7
    assert abs(o.frustum_clamp - 1.3) < 1e-7 and o.key_capacity == 0


def test_struct_layouts_match_header(tmp_path, built):
    """Compile a C probe against the header and compare sizeof/offsetof with ctypes."""
    from paper_2509_17513_b300 import _abi
    probe = tmp_path / "probe.c"
    fields = {"gc_options": _abi.Options, "gc_gaussians": _abi.Gaussians, "gc_motion": _abi.Motion,
              "gc_camera": _abi.Camera, "gc_grads": _abi.Grads, "gc_stats": _abi.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', 'int main(void) {']
    for cname, cls in fields.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-o", str(exe), str(probe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, cls in fields.items():
        assert int(got[cname]) == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_no_gpu_means_loud_failure_not_fallback(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_17513_b300 import Renderer, GCError
    with pytest.raises(GCError):
        Renderer(0)
