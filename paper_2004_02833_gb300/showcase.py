"""The reactor-like showcase (Section 5.2) as a P_N convergence study on one GPU.

The paper computes its rod geometry with P_3, P_7, P_19, P_29 and P_39 and reads off that P_19 is
already resolved (the profiles for N >= 19 agree).  ``reactor_convergence`` runs the synthetic
stand-in (``synth.reactor_like``) at each order through the C ABI, from a zero state to time t, and
reports for each N the relative difference of its u_0 field from that of the highest order, over
the whole cube and along the x-line through the rods at mid height, with the time per step.

    python -m paper_2004_02833_gb300.showcase --n 64 --steps 100
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import rtpn, synth


def reactor_convergence(n: int = 64, orders=(3, 7, 19, 29, 39), steps: int = 100,
                        precision: str = "fp32") -> dict:
    fields, per_step = {}, {}
    for N in orders:
        inst = synth.reactor_like(N, n)
        with rtpn.Context(N, inst.shape, inst.h, inst.bc, precision, inst.dt) as ctx:
            ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
            ctx.step(1)  # builds the cached launch graphs
            ctx.synchronize()
            ctx.zero_moments()
            t0 = time.perf_counter()
            ctx.step(steps)
            ctx.synchronize()
            per_step[N] = (time.perf_counter() - t0) / steps * 1e3
            fields[N] = ctx.get_component(0)
            kernel = {1: "generic", 2: "window", 3: "stage", 4: "fused"}[ctx.info().kernel]
        per_step[N] = {"ms_per_step": per_step[N], "kernel": kernel}
    top = max(orders)
    ref = fields[top]
    mid = n // 2
    line_ref = ref[mid, mid]
    out = {"workload": f"reactor-like cube {n}^3, h = 0.2, vacuum, {steps} steps (t = "
                       f"{steps * 0.3 * 0.2:.1f}), {precision}",
           "reference_order": top, "orders": {}}
    for N in orders:
        u = fields[N]
        out["orders"][N] = {
            **per_step[N],
            "rel_l2_vs_ref": float(np.linalg.norm(u - ref) / np.linalg.norm(ref)),
            "rel_max_line_vs_ref": float(np.abs(u[mid, mid] - line_ref).max() / np.abs(line_ref).max()),
            "u0_total": float(u.sum()),
        }
    out["log10_u0_line_ref"] = [float(v) for v in np.log10(np.maximum(np.abs(line_ref), 1e-30))]
    return out


def main():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--n", type=int, default=64)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--orders", default="3,7,19,29,39")
    p.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp64"])
    a = p.parse_args()
    res = reactor_convergence(a.n, tuple(int(x) for x in a.orders.split(",")), a.steps, a.precision)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
