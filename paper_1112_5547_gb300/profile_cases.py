"""Small fixed workloads for profiling the kernels under ncu.

Each case builds its lattices, runs a few steps with a fixed launch shape and
exits; the summaries under profiles/ name the exact command.

    python -m paper_1112_5547_gb300.profile_cases step   --L 512 --precision f32 --tile 22 --zchunk 64 --steps 3
    python -m paper_1112_5547_gb300.profile_cases solo_vs_batch --L 192 --tile 18 --batch-tile 3 --zchunk 32
    python -m paper_1112_5547_gb300.profile_cases ragged --batch-tile 5 --zchunk 16 --steps 3
    python -m paper_1112_5547_gb300.profile_cases step2d --L 4096 --tile 3 --steps 3
    python -m paper_1112_5547_gb300.profile_cases pfm --L 256 --steps 3

step: one D3Q19 drop lattice (R = L/4, G rho_tot = 2.4, tau = 1), `steps`
solo steps; step2d: the same on an L^2 D2Q9 lattice.  solo_vs_batch: the
same lattice stepped twice alone, then twice as a batch of one.  ragged: the
64-lattice ragged batch of inputs.ragged_drop_specs, `steps` batched steps.
pfm: the phase-field solver (FP32) on an L^3 drop (rho_A 1.2 / rho_B 0.2,
tau 0.6, g 0.3, dt 0.1), `steps` steps.
"""
from __future__ import annotations

import argparse

import numpy as np

from . import inputs, lbm_sc

G = 2.4 / inputs.RHO_TOT


def _drop_lattice(L, precision, stream):
    rA, rB = inputs.drop((L, L, L), L / 4, seed=2, dtype=np.float32)
    ref = (0.52, 0.52) if precision in ("bf16", "f16") else (0.0, 0.0)
    return lbm_sc.Lattice(lbm_sc.LBM_D3Q19, (L, L, L), 1.0, 1.0, G, precision, ref[0], ref[1],
                          stream=stream).init(rA, rB)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=["step", "step2d", "solo_vs_batch", "ragged", "pfm"])
    ap.add_argument("--L", type=int, default=192)
    ap.add_argument("--precision", default="f32", choices=list(lbm_sc.PRECISIONS))
    ap.add_argument("--tile", type=int, default=22)
    ap.add_argument("--batch-tile", type=int, default=5)
    ap.add_argument("--zchunk", type=int, default=0)
    ap.add_argument("--steps", type=int, default=3)
    a = ap.parse_args(argv)

    import torch
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        if a.case == "pfm":
            from . import phase_field
            rA, rB = inputs.drop((a.L,) * 3, a.L / 4, rho_hi=1.2, rho_lo=0.2, seed=2, dtype=np.float32)
            s = phase_field.PFM((a.L,) * 3, 1.4, 0.6, 0.3, 0.1, "f32", stream=st).init(rA - rB)
            s.step(a.steps)
        elif a.case == "step2d":
            rA, rB = inputs.drop((a.L, a.L), a.L / 4, seed=0, dtype=np.float32)
            lat = lbm_sc.Lattice(lbm_sc.LBM_D2Q9, (a.L, a.L), 1.0, 1.0, G, a.precision, stream=st).init(rA, rB)
            lat.set_tuning(a.tile, 0)
            lat.step(a.steps)
        elif a.case == "step":
            lat = _drop_lattice(a.L, a.precision, st)
            lat.set_tuning(a.tile, a.zchunk)
            lat.step(a.steps)
        elif a.case == "solo_vs_batch":
            lat = _drop_lattice(a.L, a.precision, st)
            lat.set_tuning(a.tile, a.zchunk)
            lat.step(2)
            b = lbm_sc.Batch([lat], tile=a.batch_tile, zchunk=a.zchunk, stream=st)
            b.step(2)
            st.synchronize()
            b.close()
        else:
            lats = []
            for sp in inputs.ragged_drop_specs():
                rA, rB = inputs.spec_fields(sp, dtype=np.float32)
                lats.append(lbm_sc.Lattice(lbm_sc.LBM_D3Q19, sp["shape"], sp["tau_A"], sp["tau_B"], sp["G"], "f32",
                                           stream=st).init(rA, rB))
            b = lbm_sc.Batch(lats, tile=a.batch_tile, zchunk=a.zchunk, stream=st)
            b.step(a.steps)
            st.synchronize()
            b.close()
        st.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
