"""Pathology and pacing scenarios of Sec. 5 on the quarter-scale synthetic
heart: left bundle-branch block (null conductivity along the left branch),
AV block with right-ventricular apex pacing, and right-atrial pacing without
a sinus beat. The CUDA path against the FP64 oracle over 200 ms, and the
scenario's expected physiology."""
import numpy as np
import pytest

import workloads as w
from gpu_common import act_error, tolerances

pytestmark = pytest.mark.gpu

OUT = (2500, 5000, 7500, 10000)   # steps of 0.02 ms


@pytest.fixture(scope="module")
def heart():
    case, g = w.whole_heart(h=w.heart_h_for_cells(25000, 0.25), scale=0.25, n_tree=1500, n_pmj=150)
    lab, _ = w.heart_regions(w.tet_centroids(case.xyz, case.tets) / g.scale)
    return case, g, lab


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    c = ep.Context()
    yield c
    c.close()


def _gpu(ctx, case, g, prec=None):
    from paper_2112_12854_b300 import ep
    nm = np.array([ps.model for ps in case.param_sets], np.uint8)[g.param_set]
    j = ep.job_from_case(ctx, case, precision=ep.EP_FP32_MIXED if prec is None else prec)
    j.attach_graph(g, node_model=nm)
    return j


def _parity(ctx, case, g):
    """Run GPU (FP32 mixed) and oracle side by side; return both."""
    import oracle
    from paper_2112_12854_b300 import ep
    tv, ta = tolerances(ep.EP_FP32_MIXED)
    o = oracle.Sim(case)
    o.attach_graph(g)
    j = _gpu(ctx, case, g)
    done, worst = 0, 0.0
    for n in OUT:
        o.run(n - done)
        j.step(n - done)
        done = n
        worst = max(worst, np.abs(j.V - o.V).max(), np.abs(j.graph_read(0) - o.graph_get(0)).max())
    assert worst <= tv, worst
    assert act_error(j.activation_times(), o.activation_times()) <= ta
    assert act_error(j.graph_activation_times(), o.graph_activation_times()) <= ta
    return j, o


def test_left_bundle_branch_block(ctx, heart):
    case, g, lab = heart
    cb, gb = w.heart_scenario(case, g, block="left")
    j, o = _parity(ctx, cb, gb)
    a_blk = o.activation_times()
    h = _gpu(ctx, case, g)
    h.step(OUT[-1])
    a_ok = h.activation_times()
    ag_blk, ag_ok = o.graph_activation_times(), h.graph_activation_times()
    lv_blk, rv_blk = np.nanmin(ag_blk[gb.lv_nodes]), np.nanmin(ag_blk[gb.rv_nodes])
    lv_ok = np.nanmin(ag_ok[g.lv_nodes])
    vent = (lab == 1) | (lab == 2)
    print("LBBB: left tree first activation %.1f ms (healthy %.1f), right tree %.1f ms; "
          "ventricles fully active at %.1f ms (healthy %.1f)"
          % (lv_blk, lv_ok, rv_blk, np.nanmax(a_blk[vent]), np.nanmax(a_ok[vent])))
    # the right branch conducts as before; the blocked left tree is reached only
    # late, antidromically from the myocardium, and the ventricles take longer
    assert lv_blk > rv_blk + 10.0 and lv_blk > lv_ok + 10.0
    assert np.isfinite(a_blk[vent]).all() and np.nanmax(a_blk[vent]) > np.nanmax(a_ok[vent]) + 3.0
    for x in (j, h):
        x.destroy()


def test_av_block_with_ventricular_pacing(ctx, heart):
    case, g, lab = heart
    cb, gb = w.heart_scenario(case, g, av_block=True)
    blk = _gpu(ctx, cb, gb)
    blk.step(OUT[-1])
    assert not np.isfinite(blk.activation_times()[(lab == 1) | (lab == 2)]).any()   # ventricles silent
    onset = 100.0
    cp, gp = w.heart_scenario(case, g, av_block=True, lead="rv_apex", lead_radius=1.0, lead_onset=onset)
    j, o = _parity(ctx, cp, gp)
    a, ag = o.activation_times(), o.graph_activation_times()
    print("pacing: ventricles activated %.2f, Purkinje nodes %.2f" %
          (np.isfinite(a[(lab == 1) | (lab == 2)]).mean(), np.isfinite(ag[gp.lv_nodes[0]:]).mean()))
    assert np.isfinite(a[(lab == 1) | (lab == 2)]).mean() > 0.5
    tree = np.concatenate([gp.lv_nodes, gp.rv_nodes])
    assert np.isfinite(ag[tree]).mean() > 0.5                  # entered antidromically through PMJs
    assert np.nanmin(ag[tree]) > onset                          # ... after the lead fired
    assert not np.isfinite(ag[gp.his]) or ag[gp.his] > onset
    for x in (j, blk):
        x.destroy()


def test_atrial_pacing_without_sinus(ctx, heart):
    case, g, lab = heart
    onset = 5.0
    cp, gp = w.heart_scenario(case, g, sinus=False, lead="ra_appendage", lead_radius=1.0, lead_onset=onset,
                              two_way=True, cn_amplitude=-1000.0, cn_duration=1.0)
    j, o = _parity(ctx, cp, gp)
    a, ag = o.activation_times(), o.graph_activation_times()
    site = w.heart_lead_site(cp, gp, "ra_appendage")
    d = np.linalg.norm(w.tet_centroids(cp.xyz, cp.tets) - site, axis=1)
    bundle = ag[:gp.n_bundle]
    print("atrial pacing: first bundle activation %.2f ms, atria activated %.2f" %
          (np.nanmin(bundle), np.isfinite(a[lab >= 3]).mean()))
    assert np.nanmin(a[d <= 1.0]) < np.nanmin(bundle)         # the lead excites the myocardium first
    assert np.isfinite(bundle).mean() > 0.8                    # ... which then excites the bundle
    assert np.isfinite(a[lab >= 3]).mean() > 0.9
    j.destroy()
