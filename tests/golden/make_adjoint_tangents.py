"""Writes adjoint_tangents_<n>.json, the reference directional derivatives of
the differentiation workload for the CUDA adjoint.

Reference: forward-mode automatic differentiation (torch.autograd.forward_ad)
through oracle/torch_stage.py, the plain-PyTorch CPU FP64 restatement of the
euler_step (Alg. 1-3) and of SSP-RK3 (Sec. 3.6, eq. ssprk3), whose forward
values are pinned to the C oracle.  Forward mode carries one tangent through
every step, so it needs no tape and gives dJ/dU^0 . v directly, including
the dependence of tau_n on the state (tau_n = c_cfl min_i m_i/(-2 d_ii)).
On the configured mesh the vortex is z-invariant away from the bumps:
z-neighbours hold bitwise equal states, min/max decisions tie exactly or are
decided by rounding, and the derivative there is not unique (Reading A33).
With --jitter 0.2 (seed 3) the nodes move off the lattice and no such ties
occur; that variant is the reference the CUDA adjoint is checked against.

Workload: the n^3 periodic isentropic vortex with eight seeded Gaussian
density bumps (amplitude 1e-2, width 0.1, seed 5; workloads.bumpy_vortex_state),
J = sum over nodes x_i in [0.4, 0.6]^3 of m_i p_i(U^N) after N SSP-RK3 steps at
CFL 0.5, directions v_k = xi_k |U^0| (workloads.perturbation_directions, seed
16).  Only oracle/ and the input generators are used.

    python tests/golden/make_adjoint_tangents.py --n 64 --steps 100 --directions 2 --jitter 0.2
    (or one direction at a time: --direction 1 adds the second to a file holding the first)
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402
import torch.autograd.forward_ad as fwAD  # noqa: E402

import oracle as O  # noqa: E402
from oracle import torch_stage as T  # noqa: E402
from paper_2007_00094_gb300 import workloads as W  # noqa: E402


def box_weights(x, mi, lo=0.4, hi=0.6):
    inside = np.all((x >= lo) & (x <= hi), axis=1)
    return np.where(inside, mi, 0.0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--directions", type=int, default=2)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--jitter", type=float, default=0.0, help="node jitter (fraction of h), seed 3; 0 = as configured")
    ap.add_argument("--out", default=None)
    ap.add_argument("--direction", type=int, default=None,
                    help="compute only direction k of the seeded set and add it to the existing --out record "
                         "(which must hold directions 0 .. k-1 of the same workload)")
    args = ap.parse_args()
    torch.set_num_threads(args.threads)
    mesh = W.vortex_mesh(args.n, jitter=args.jitter, seed=3) if args.jitter > 0 else W.vortex_mesh(args.n)
    U0 = W.bumpy_vortex_state(mesh)
    om = O.assemble(mesh)
    tm = T.TorchMesh(om)
    w = torch.as_tensor(box_weights(mesh.x, om.mi))
    dirs = W.perturbation_directions(U0, args.directions, seed=16)
    out = args.out or os.path.join(HERE, f"adjoint_tangents_{args.n}.json")
    rec = {"source": "forward-mode AD through oracle/torch_stage.py (make_adjoint_tangents.py)",
           "workload": f"bumpy vortex {args.n}^3 periodic, 8 bumps amplitude 1e-2 width 0.1 seed 5",
           "functional": "sum over x_i in [0.4,0.6]^3 of m_i p_i(U^N) (oracle lumped masses)",
           "jitter": args.jitter, "mesh_seed": 3 if args.jitter > 0 else None,
           "n": args.n, "steps": args.steps, "cfl": 0.5, "directions_seed": 16, "J": None, "dJ_dv": [],
           "seconds": []}
    todo = list(enumerate(dirs))
    if args.direction is not None:
        with open(out) as fh:
            prev = json.load(fh)
        for key in ("n", "steps", "jitter", "mesh_seed", "directions_seed"):
            assert prev[key] == rec[key], key
        assert len(prev["dJ_dv"]) == args.direction, "directions must be added in order"
        rec = prev
        todo = [(args.direction, dirs[args.direction])]
    for k, v in todo:
        t0 = time.perf_counter()
        with fwAD.dual_level():
            U = fwAD.make_dual(torch.as_tensor(U0), torch.as_tensor(v))
            for _ in range(args.steps):
                U, _ = T.ssprk3_step(tm, U)
            J = (w * T.pressure(U)).sum()
            val, tan = fwAD.unpack_dual(J)
        rec["J"] = float(val)
        rec["dJ_dv"].append(float(tan))
        rec["seconds"].append(time.perf_counter() - t0)
        tmp = out + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(rec, fh, indent=1)
        os.replace(tmp, out)
        print(f"direction {k}: dJ.v = {float(tan):.16e} ({rec['seconds'][-1]:.0f} s)", flush=True)


if __name__ == "__main__":
    main()
