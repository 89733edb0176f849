"""Render the interface phi = 0 of a workload to a PPM image (headless, on the GPU).

python -m paper_2406_01322_gb300.render --workload channel_128x128x129 --steps 20 --out drops.ppm
"""
import argparse
import math

import torch

from . import binding, inputs


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="channel_128x128x129", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--steps", type=int, default=0, help="time steps before the image")
    ap.add_argument("--width", type=int, default=960)
    ap.add_argument("--height", type=int, default=540)
    ap.add_argument("--fov", type=float, default=45.0)
    ap.add_argument("--out", default="interface.ppm")
    a = ap.parse_args(argv)
    w = dict(inputs.WORKLOADS[a.workload])
    lx, ly = 4 * math.pi, 2 * math.pi
    g = binding.Grid(w["nx"], w["ny"], w["nz"], re_tau=w["re_tau"], we=w["we"], ch=w["ch"],
                     pe=w["pe"], dt=w["dt"], precision=w["precision"])
    g.set_fields(*[torch.from_numpy(f) for f in inputs.initial_fields(**w)])
    g.step(a.steps)
    rgb, _ = g.render_interface(a.width, a.height, (-0.3 * lx, -0.8 * ly, 2.5),
                                (0.5 * lx, 0.5 * ly, 0.0), (0.0, 0.0, 1.0), a.fov)
    binding.write_ppm(a.out, rgb)
    print(f"wrote {a.out} ({a.width}x{a.height}, {a.workload}, step {a.steps})")


if __name__ == "__main__":
    main()
