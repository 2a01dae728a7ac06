"""Stochastic estimate of the disconnected loop Tr[gamma5 M^-1] (the paper's production use).

For Z2 noise vectors eta_n (tm_noise_z2, counter-based, source n uses seed0 + n) the batched
solver gives s_n = M^-1 eta_n on both parities (even-odd solve of eq. 2.2 + reconstruction of
eq. 2.4), and each source contributes eta_n^dag gamma5 s_n (tm_g5dot on each parity).  The
estimate is the mean over sources; its standard error is the sample standard deviation over
sqrt(N).  Every step runs in the library's kernels; this module only loops over batches.
"""
from __future__ import annotations

import time

import numpy as np

from . import (TM_PC_ASYM, TM_PREC_F32, TM_PREC_F64, Field, g5dot, noise_z2, prepare_rhs, reconstruct_odd,
               solve_multi)


def g5_trace(gauge, nsources=256, batch=16, seed0=3000, tol=1e-8, solver="mixed", sloppy_prec=TM_PREC_F32,
             use_graph=True, pc=TM_PC_ASYM, return_solutions=False, true_prec=TM_PREC_F64):
    import torch
    vals, iters, t_solve = [], [], 0.0
    sols = []
    for b0 in range(0, nsources, batch):
        nb = min(batch, nsources - b0)
        ee, eo = Field(gauge, TM_PREC_F64, nb), Field(gauge, TM_PREC_F64, nb)
        noise_z2(gauge, ee, 0, seed0 + b0)
        noise_z2(gauge, eo, 1, seed0 + b0)
        bp, xe, xo = Field(gauge, TM_PREC_F64, nb), Field(gauge, TM_PREC_F64, nb), Field(gauge, TM_PREC_F64, nb)
        torch.cuda.synchronize()
        t0 = time.time()
        prepare_rhs(gauge, bp, ee, eo, pc, False)
        _, stats = solve_multi(gauge, xe, bp, solver=solver, sloppy_prec=sloppy_prec, tol=tol, pc=pc,
                               use_graph=use_graph, true_prec=true_prec)
        reconstruct_odd(gauge, xo, eo, xe, False)
        torch.cuda.synchronize()
        t_solve += time.time() - t0
        vals.extend(list(g5dot(gauge, ee, xe) + g5dot(gauge, eo, xo)))
        iters.extend(s["iterations"] for s in stats)
        if return_solutions and b0 == 0:  # the first batch only (a 32^3x64 batch of 16 is 6.4 GB)
            sols.append((xe, xo))
    v = np.array(vals)
    out = {"estimate": complex(v.mean()), "stderr": float(np.sqrt(v.real.var(ddof=1) + v.imag.var(ddof=1))
                                                           / np.sqrt(len(v))) if len(v) > 1 else float("nan"),
           "per_source": v, "iterations": iters, "solve_seconds": t_solve,
           "solves_per_second": len(v) / t_solve if t_solve > 0 else float("nan")}
    if return_solutions:
        out["solutions"] = sols
    return out
