"""Command line: render one scene of the synthetic workloads on cuda:0.

    python -m paper_1012_5107_gb300 render [--workload small|main|hd|gauss]
        [--kind mirror|bare|cloak] [--precision fp32|fp64]
        [--integrator rk4|dp45|rk4t] [--side N | --width W --height H] [--spp S]
        [--extent E] [--amplitude A] [--centre-line] [--variant V] [--min-active M]
        [--autotune] [--warmup W] [--repeat K] [--ppm out.ppm]

Builds nothing: the CUDA library must have been built (python -c 'import
__graft_entry__ as g; g.build()').  Each render is one launch through
rt_render; the time is measured with CUDA events on the launching stream after
`--warmup` untimed renders.  Prints one JSON line (time per render, rays,
integrator steps, Mrays/s, G steps/s) and optionally writes the 8-bit image as
a binary PPM.
"""
from __future__ import annotations

import argparse
import json
import sys

from . import inputs

INTEGRATORS = {"rk4": inputs.RK4, "dp45": inputs.DP45, "rk4t": 2}


def scene_params(args) -> tuple[dict, object]:
    prec = inputs.FP32 if args.precision == "fp32" else inputs.FP64
    tex = None
    if args.workload == "small":
        base = inputs.config_small(precision=prec)
    elif args.workload == "main":
        base = inputs.config_main(precision=prec)
    elif args.workload == "hd":
        base = inputs.config_hd(extent=args.extent or 8.0, A=args.amplitude or 0.04, precision=prec)
        tex = inputs.value_noise(base["tex_size"], seed=3)
    else:
        base = inputs.gauss_scene(width=512, height=512, spp=4, seed=2, precision=prec)
    renders = inputs.gauss_renders(base) if args.workload == "gauss" else inputs.three_renders(base)
    p = dict(renders[args.kind])
    if args.side:
        p["width"] = p["height"] = args.side
    if args.width:
        p["width"] = args.width
    if args.height:
        p["height"] = args.height
    if args.spp:
        p["spp"] = args.spp
    if args.extent and args.workload != "hd":
        p["E"] = args.extent
    if args.amplitude is not None and args.workload != "hd":
        p["A"] = args.amplitude
    if args.integrator:
        p["integrator"] = INTEGRATORS[args.integrator]
        if p["integrator"] == inputs.DP45 and args.workload != "hd":
            tol = 1e-5 if prec == inputs.FP32 else 1e-7
            p["rtol"] = p["atol"] = tol
    if args.centre_line:
        p["centre_line"] = 1
    return p, tex


def write_ppm(path: str, img) -> None:
    h, w, _ = img.shape
    with open(path, "wb") as f:
        f.write(b"P6\n%d %d\n255\n" % (w, h))
        f.write(img.tobytes())


def cmd_render(args) -> int:
    import torch

    from . import rt
    torch.cuda.set_device(0)
    p, tex = scene_params(args)
    sc = rt.Scene(p, tex=tex)
    rgb = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
    rgb8 = torch.zeros(sc.shape, dtype=torch.uint8, device="cuda")
    if args.variant is not None or args.min_active:
        sc.set_launch(-1 if args.variant is None else args.variant, args.min_active or 0)
    if args.autotune:
        sc.autotune(rgb, trials=1)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            sc.render(rgb, rgb8, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.repeat):
            sc.render(rgb, rgb8, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.repeat, 1)
    st = sc.stats()
    out = {"workload": args.workload, "kind": args.kind, "precision": args.precision,
           "width": sc.width, "height": sc.height, "out_width": sc.wout, "spp": sc.spp,
           "integrator": int(p["integrator"]), "ms": round(ms, 4), "rays": st["rays"], "steps": st["steps"],
           "Mrays_per_s": round(st["rays"] / (ms * 1e-3) / 1e6, 3) if ms > 0 else None,
           "Gsteps_per_s": round(st["steps"] / (ms * 1e-3) / 1e9, 4) if ms > 0 else None,
           "newton_per_step": round(st["newton"] / st["steps"], 3) if st["steps"] else None,
           "sched_timeouts": st["sched_timeouts"], "launch": sc.get_launch()}
    if args.ppm:
        write_ppm(args.ppm, rgb8.cpu().numpy())
        out["ppm"] = args.ppm
    print(json.dumps(out), flush=True)
    sc.close()
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_1012_5107_gb300")
    sub = ap.add_subparsers(dest="cmd", required=True)
    r = sub.add_parser("render", help="render one scene and time it")
    r.add_argument("--workload", default="main", choices=["small", "main", "hd", "gauss"])
    r.add_argument("--kind", default="cloak", choices=["mirror", "bare", "cloak"])
    r.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    r.add_argument("--integrator", choices=sorted(INTEGRATORS))
    r.add_argument("--side", type=int)
    r.add_argument("--width", type=int)
    r.add_argument("--height", type=int)
    r.add_argument("--spp", type=int)
    r.add_argument("--extent", type=float)
    r.add_argument("--amplitude", type=float)
    r.add_argument("--centre-line", action="store_true")
    r.add_argument("--variant", type=int, help="launch variant: 0-2 the per-lane loop, 3 the wavefront loop")
    r.add_argument("--min-active", type=int, default=0, help="lanes inside the cloak that keep a warp integrating")
    r.add_argument("--autotune", action="store_true", help="time the launch configurations first and keep the fastest")
    r.add_argument("--warmup", type=int, default=1)
    r.add_argument("--repeat", type=int, default=3)
    r.add_argument("--ppm")
    args = ap.parse_args(argv)
    if args.cmd == "render":
        return cmd_render(args)
    return 2


if __name__ == "__main__":
    sys.exit(main())
