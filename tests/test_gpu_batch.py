"""The batching workload (C4) through one plan: 512 BF16 stream matrices of
uneven size, m log-uniform in [256, 4096], n in [256, 2048], k in {10, 20,
40}, r = k / 2, each with its own sketch (problem 1.1 is solved per matrix,
Section 1).

Sizes are not rounded, so most contiguous BF16 rows do not start on 16-byte
boundaries: the plan copies those matrices to aligned rows in its workspace
at every execution, and every matrix takes the tensor-core kernel
(TSK_KERNEL_TC accepts both layouts).  Stored with a padded leading
dimension, nothing is copied.  Sampled outputs are compared with the oracle
at the 1e-3 gap; every ||A||^2 is compared with the oracle's sum of
squares.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
GAP = 1e-3


@pytest.fixture(scope="module")
def tsk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2209_14637_gb300 as mod
    from paper_2209_14637_gb300 import build
    build.build()
    return mod


@pytest.fixture(scope="module")
def batch():
    items = synth.ragged_sizes(512)
    Ss = [synth.item_sketch(it, device="cuda") for it in items]
    return items, Ss


def _np(t):
    return t.detach().double().cpu().numpy()


def _sample(items, per_k=8):
    """Indices spread over the three k values, smallest and largest m first."""
    idx = []
    for k in (10, 20, 40):
        ids = sorted((i for i, it in enumerate(items) if it.k == k),
                     key=lambda i: items[i].m * items[i].n)
        pick = np.linspace(0, len(ids) - 1, per_k).round().astype(int)
        idx += [ids[j] for j in pick]
    return sorted(set(idx))


@pytest.mark.parametrize("pad_rows", [False, True])
def test_c4_ragged_batch_of_512(tsk, batch, pad_rows):
    items, Ss = batch
    As = synth.ragged_batch(items, device="cuda", pad_rows=pad_rows)
    rs = [it.r for it in items]
    unaligned = sum((A.stride(0) * 2) % 16 != 0 for A in As)
    if pad_rows:
        assert unaligned == 0
    else:
        assert unaligned > 256  # most rows start off a 16-byte boundary
    h = tsk.Handle(kernel=tsk.KERNEL_TC, refine_q=tsk.REFINE_ALWAYS)
    err = torch.empty(len(As), dtype=torch.float64, device="cuda")
    nrm = torch.empty(len(As), dtype=torch.float64, device="cuda")
    plan = h.plan(As, Ss, rs, err, nrm)
    plan.execute()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    e = _np(err)
    assert np.isfinite(e).all() and (e > 0).all()
    for i, A in enumerate(As):
        np.testing.assert_allclose(float(nrm[i]), float(np.sum(_np(A) ** 2)), rtol=1e-6)
    for i in _sample(items):
        o = oracle.scw(_np(As[i]), _np(Ss[i]), rs[i], dense=False)
        assert abs(e[i] - o["err"]) <= GAP * o["err"], (i, items[i], e[i], o["err"])
    # a second execution of the same graph gives the same errors
    plan.execute()
    torch.cuda.synchronize()
    np.testing.assert_allclose(_np(err), e, rtol=1e-12)
    plan.close()
    h.close()


def test_autotune_then_the_tuned_plan_matches_the_oracle(tsk, batch, tmp_path):
    """The autotuner times both cluster shapes for each size class of the
    batch that has two (256 < m <= 2048), keeps the faster in the handle and
    round-trips it through JSON; plans built afterwards use it and still
    match the oracle, and a second handle that loads the file builds the
    same plan (same errors, bit for bit)."""
    import json
    items, Ss = batch
    As = synth.ragged_batch(items[:96], device="cuda", pad_rows=True)
    S96, r96 = Ss[:96], [it.r for it in items[:96]]
    h = tsk.Handle(kernel=tsk.KERNEL_TC, refine_q=tsk.REFINE_ALWAYS)
    h.autotune(As, S96, r96, reps=3)
    path = tmp_path / "tune.json"
    h.autotune_save(str(path))
    table = json.loads(path.read_text())
    assert table["classes"], table
    for c in table["classes"]:
        assert c["rows_per_cta"] in (256, 384, 512)
        timed = {s: c[f"us_per_matrix_{s}"] for s in (512, 256, 384)
                 if c[f"us_per_matrix_{s}"] > 0}
        assert 512 in timed
        assert c["rows_per_cta"] == min(timed, key=timed.get)
    out = h.approx_batch(As, S96, r96)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    e = _np(out["err"])
    for i in _sample(items[:96], per_k=3):
        o = oracle.scw(_np(As[i]), _np(S96[i]), r96[i], dense=False)
        assert abs(e[i] - o["err"]) <= GAP * o["err"], (i, items[i])
    h2 = tsk.Handle(kernel=tsk.KERNEL_TC, refine_q=tsk.REFINE_ALWAYS)
    h2.autotune_load(str(path))
    e2 = _np(h2.approx_batch(As, S96, r96)["err"])
    np.testing.assert_allclose(e2, e, rtol=1e-12)
    h.close()
    h2.close()
