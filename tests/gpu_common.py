"""Shared helpers of the GPU tests: tolerances, a library context, and
runners that produce the oracle's and the CUDA path's outputs on the same
seeded inputs."""
import numpy as np
import pytest

import workloads as w

# Tolerances (stated per result):
#  - FP32 mixed vs FP64 oracle: |dV| <= 1 mV at every output time, activation
#    time within 0.5 ms at every cell (the contract of the FP32 path);
#  - FP64 plain vs FP64 oracle: same arithmetic up to rounding order and libm
#    differences (<= 2 ulp per call): |dV| <= 1e-6 mV, |dt_act| <= 1e-6 ms.
TOL_V_MIXED, TOL_ACT_MIXED = 1.0, 0.5
TOL_V_PLAIN, TOL_ACT_PLAIN = 1e-6, 1e-6


def tolerances(precision):
    from paper_2112_12854_b300 import ep
    return (TOL_V_PLAIN, TOL_ACT_PLAIN) if precision == ep.EP_FP64_PLAIN else (TOL_V_MIXED, TOL_ACT_MIXED)


def act_error(a, b):
    fa, fb = np.isfinite(a), np.isfinite(b)
    assert np.array_equal(fa, fb), f"{np.sum(fa != fb)} cells activated on one side only"
    return float(np.abs(a[fa] - b[fa]).max()) if fa.any() else 0.0


def run_oracle(case, outputs):
    import oracle
    s = oracle.Sim(case)
    res = {}
    done = 0
    for n in outputs:
        s.run(n - done)
        done = n
        res[n] = s.V
    return res, s.activation_times(), s


def run_gpu(ctx, case, outputs, precision):
    from paper_2112_12854_b300 import ep
    j = ep.job_from_case(ctx, case, precision=precision)
    res = {}
    done = 0
    for n in outputs:
        j.step(n - done)
        done = n
        res[n] = j.V
    return res, j.activation_times(), j


def isolated_cells(models_variants, amp=-52.0):
    """One isolated tet per (model, variant): no shared faces, so each cell is
    a single-cell model run through the tissue path."""
    k = len(models_variants)
    base = np.array([[0, 0, 0], [0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5]], float)
    xyz = np.concatenate([base + [2.0 * i, 0, 0] for i in range(k)])
    tets = np.arange(4 * k, dtype=np.int32).reshape(k, 4)
    sets = [w.ParamSet(model=m, variant=v) for m, v in models_variants]
    case = w.TissueCase("cells", xyz, tets, w.fibres_uniform(k), np.arange(k, dtype=np.uint8),
                        np.ones(k, np.uint8), sets, [w.Stimulus(amp, 0.0, 1.0, 500.0)], 0.02, 0, 0.0)
    return case
