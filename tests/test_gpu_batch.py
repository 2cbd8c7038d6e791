"""Batched CUDA-graph launch of uneven plans and the schedule autotuner."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2512_18863_gb300 import synth as S
from paper_2512_18863_gb300.batch import DoseBatch
from paper_2512_18863_gb300.engine import DoseEngine

pytestmark = pytest.mark.gpu


def _plans():
    return [S.small_pelvis(seed=50 + q, n=n, spacing=sp, n_cp=c, r_px=r)
            for q, (n, sp, c, r) in enumerate([((20, 32, 36), 3.0, 7, 5), ((16, 28, 28), 4.0, 3, 4),
                                               ((24, 40, 40), 3.0, 11, 6), ((18, 30, 26), 3.0, 5, 8)])]


def test_batch_matches_individual_calls_and_oracle():
    ws = _plans()
    engines = [DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso) for w in ws]
    rng = np.random.default_rng(1)
    grads = [rng.standard_normal(w.phantom.shape).astype(np.float32) for w in ws]
    b = DoseBatch(engines, [w.plan.leaves for w in ws], [w.plan.jaws for w in ws],
                  [w.plan.mu for w in ws], grads, n_branches=3)
    for _ in range(2):                      # the graph can be replayed
        b.launch()
    t = b.plan_times_ms()
    assert t.shape == (4,) and np.all(t > 0)
    assert b.kernels > 0
    for i, (w, e) in enumerate(zip(ws, engines)):
        full = e.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).clone()
        # the pass size only regroups the sum over control points
        assert torch.allclose(b.dose[i], full, rtol=0, atol=1e-6 * float(full.max()))
        assert 1 <= b.pass_cp[i] <= e.info["chunk_cp"]
        e.set_chunk(b.pass_cp[i])
        d = e.forward(w.plan.leaves, w.plan.jaws, w.plan.mu)
        dl, dj, dm = e.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, grads[i])
        assert torch.equal(b.dose[i], d)
        assert torch.equal(b.dleaves[i], dl) and torch.equal(b.djaws[i], dj) and torch.equal(b.dmu[i], dm)
    ref = O.Model(ws[2].phantom, ws[2].machine, ws[2].plan).dose()
    got = b.dose[2].cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-4 * ref.max()
    b.close()
    for e in engines:
        e.close()


def test_uneven_eight_plan_batch_in_rounds_matches_individual_calls_and_oracle():
    """Eight uneven plans cut into 1-4 passes each: the batch runs in rounds
    (round c holds pass c of every plan that has one, so plans drop out of the
    later rounds), each round one shared FFT launch and one shared gather
    launch per direction over the plans still in it. Every plan equals its
    own calls with the same pass size bit for bit (dose and gradients); two
    plans match the oracle."""
    shapes = [((20, 32, 36), 3.0, 9, 5, 3), ((16, 28, 28), 4.0, 3, 4, 3), ((24, 40, 40), 3.0, 12, 6, 3),
              ((18, 30, 26), 3.0, 5, 8, 2), ((22, 36, 30), 3.0, 8, 5, 8), ((16, 24, 40), 3.5, 6, 3, 2),
              ((20, 34, 34), 3.0, 10, 7, 4), ((14, 26, 30), 4.0, 4, 4, 1)]
    ws = [S.small_pelvis(seed=70 + q, n=n, spacing=sp, n_cp=c, r_px=r)
          for q, (n, sp, c, r, _) in enumerate(shapes)]
    engines = [DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso) for w in ws]
    for e, sh in zip(engines, shapes):
        e.set_chunk(sh[4])
    rng = np.random.default_rng(8)
    grads = [rng.standard_normal(w.phantom.shape).astype(np.float32) for w in ws]
    b = DoseBatch(engines, [w.plan.leaves for w in ws], [w.plan.jaws for w in ws],
                  [w.plan.mu for w in ws], grads, n_branches=4)
    b.launch()
    b.launch()
    passes = [-(-w.plan.n_cp // pc) for w, pc in zip(ws, b.pass_cp)]
    assert b.pass_cp == [sh[4] for sh in shapes] and min(passes) == 1 and max(passes) == 4
    for i, (w, e) in enumerate(zip(ws, engines)):
        d = e.forward(w.plan.leaves, w.plan.jaws, w.plan.mu)
        dl, dj, dm = e.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, grads[i])
        assert torch.equal(b.dose[i], d), i
        assert torch.equal(b.dleaves[i], dl) and torch.equal(b.djaws[i], dj) and torch.equal(b.dmu[i], dm), i
    for i in (0, 6):
        mod = O.Model(ws[i].phantom, ws[i].machine, ws[i].plan)
        ref = mod.dose()
        got = b.dose[i].cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 1e-4 * ref.max()
        for gg, rr in zip((b.dleaves[i], b.djaws[i], b.dmu[i]), mod.dose_grad(grads[i].astype(np.float64))):
            gg = gg.cpu().numpy().astype(np.float64)
            assert np.abs(gg - rr).max() <= 1e-3 * np.abs(rr).max()
    b.close()
    for e in engines:
        e.close()


def test_batch_mixes_convolution_paths_and_fft_size_limits():
    """One batched FFT launch per round serves plans with different size
    limits (a small limit sends slices to the tensor-core overflow pass) while
    tensor-core and SIMT plans run their own kernels on their branches; every
    result equals the plan's individual call at the batch's pass size bit for
    bit."""
    ws = _plans()
    paths = [("fft", 32), ("tc", None), ("fft", None), ("simt", None)]
    engines = [DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso, conv=c, fft_pmax=pm)
               for w, (c, pm) in zip(ws, paths)]
    assert engines[0].info["fft_pmax"] == 32 and engines[1].info["fft_pmax"] == 0
    rng = np.random.default_rng(2)
    grads = [rng.standard_normal(w.phantom.shape).astype(np.float32) for w in ws]
    grads[1] = None                         # forward only for one plan
    b = DoseBatch(engines, [w.plan.leaves for w in ws], [w.plan.jaws for w in ws],
                  [w.plan.mu for w in ws], grads, n_branches=2)
    b.launch()
    b.launch()
    b.plan_times_ms()
    for i, (w, e) in enumerate(zip(ws, engines)):
        e.set_chunk(b.pass_cp[i])
        d = e.forward(w.plan.leaves, w.plan.jaws, w.plan.mu)
        assert torch.equal(b.dose[i], d), i
        if grads[i] is not None:
            dl, dj, dm = e.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, grads[i])
            assert torch.equal(b.dleaves[i], dl) and torch.equal(b.djaws[i], dj) and torch.equal(b.dmu[i], dm), i
    b.close()
    for e in engines:
        e.close()


def test_autotune_keeps_results_and_picks_a_schedule():
    w = _plans()[2]
    e = DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso, scratch_budget_bytes=64 << 20)
    ref = e.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).clone()
    g = np.ones(w.phantom.shape, np.float32)
    r = e.autotune(w.plan.leaves, w.plan.jaws, w.plan.mu, g)
    assert r["n_candidates"] >= 2 and r["best_ms"] > 0
    assert 1 <= r["chunk_cp"] <= w.plan.n_cp
    assert e.info["chunk_cp"] == r["chunk_cp"] and e.info["tensor_cores"] == r["tensor_cores"]
    if r["tensor_cores"]:
        # the chosen tile shape (phase depth) is live on the plan
        assert all(1 <= ph <= 4 for ph in r["phase"])
        assert e.info["tc_ctas_per_sm"] == r["tc_ctas_per_sm"] and min(r["tc_ctas_per_sm"]) >= 1
    d = e.forward(w.plan.leaves, w.plan.jaws, w.plan.mu)
    assert torch.allclose(d, ref, rtol=0, atol=1e-5 * float(ref.max()))
    e.close()


def test_every_tensor_core_tile_shape_gives_the_same_dose():
    """Each phase depth the autotuner may pick (1..4 kernel rows per operand
    buffer, per direction) computes the same dose and gradients."""
    from paper_2512_18863_gb300 import _lib
    w = _plans()[0]
    e = DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso)
    g = np.random.default_rng(3).standard_normal(w.phantom.shape).astype(np.float32)
    ref = e.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).clone()
    rg = [t.clone() for t in e.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, g)]
    for ph in (1, 2, 3, 4):
        _lib.pdrt_plan_set_tc_phase(e._plan, ph, ph)
        d = e.forward(w.plan.leaves, w.plan.jaws, w.plan.mu)
        assert torch.allclose(d, ref, rtol=0, atol=1e-5 * float(ref.max())), ph
        for a, b in zip(e.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, g), rg):
            assert torch.allclose(a, b, rtol=0, atol=1e-4 * float(b.abs().max())), ph
    e.close()
