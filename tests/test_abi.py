"""The C ABI library loads and exports every entry point declared in
include/*.h; descriptor validation runs on the host (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

from paper_1012_5107_gb300 import build as B
from paper_1012_5107_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rt():
    B.build()
    from paper_1012_5107_gb300 import rt as r
    r.lib()
    return r


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(rt_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_function(rt):
    names = declared_functions()
    assert "rt_render" in names and "rt_create_scene" in names
    lib = rt.lib()
    for n in names:
        assert hasattr(lib, n), n
        getattr(lib, n)
    assert set(rt.EXPORTS) <= set(names)


def test_version(rt):
    assert "sm_103a" in rt.version()


@pytest.mark.parametrize("bad,field", [
    (dict(Lambda=0.0), "Lambda"), (dict(A=0.2), "A must"), (dict(width=0), "width"),
    (dict(hfov_deg=180.0), "hfov"), (dict(H=0.05), "H > 2A"), (dict(integrator=7), "integrator"),
    (dict(integrator=3), "integrator"),
    (dict(precision=3), "precision"), (dict(background=1, tex_size=0), "texture"),
    (dict(mirror=0, cloak=1), "trochoid"), (dict(flags=8), "unknown bits"), (dict(max_steps=0), "max_steps"),
    (dict(flags=2), "plate lies on the flat mirror"),
    (dict(mirror=2, A=0.3, gauss_w=0.306, H=1.1), "0.8 gauss_w"), (dict(mirror=2, gauss_w=0.0), "gauss_w"),
    (dict(mirror=2, A=0.13, gauss_w=0.306, H=1.1, flags=4), "no options"), (dict(mirror=3), "mirror must"),
])
def test_invalid_descriptor_is_rejected(rt, bad, field):
    p = inputs.base_scene(**bad)
    with pytest.raises(rt.RtError) as e:
        rt.Scene(p)
    assert e.value.code == rt.RT_EINVAL
    assert field in str(e.value)


def test_struct_layouts_match_header(rt, tmp_path):
    """Offsets of every ctypes field equal the C compiler's for include/rt.h."""
    import subprocess
    structs = {"rt_scene_desc": rt.SceneDesc, "rt_ray_record": rt.RayRecord, "rt_stats": rt.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rt.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_validate_desc_on_host(rt):
    rt.validate(inputs.base_scene())
    rt.validate(inputs.base_scene(integrator=2))          # RK4 in physical time (Eq. 11)
    rt.validate(inputs.gauss_scene())                     # the Gaussian conformal cloak (Fig. 4)
    with pytest.raises(rt.RtError) as e:
        rt.validate(inputs.base_scene(spp=0))
    assert e.value.code == rt.RT_EINVAL


@pytest.mark.parametrize("over", [dict(width=64, height=48, spp=4), dict(width=33, height=17, spp=1, centre_line=1),
                                  dict(width=256, height=256, spp=64)])
def test_request_bytes(rt, over):
    """A request's footprint in a server budget: 76 bytes per sample (ray state
    and a colour slot) and 16 per pixel (output colour and a sample counter)."""
    p = inputs.base_scene(**over)
    wout = 1 if p["centre_line"] else p["width"]
    assert rt.request_bytes(p) == p["height"] * wout * (76 * p["spp"] + 16)


def test_request_bytes_rejects_invalid(rt):
    with pytest.raises(rt.RtError) as e:
        rt.request_bytes(inputs.base_scene(width=0))
    assert e.value.code == rt.RT_EINVAL
