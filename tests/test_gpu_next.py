"""Two experiments of the paper on the GPU path, against the oracle.

* Classical SCW with data-oblivious sketches (Section 1: a Gaussian or a
  sign matrix S): the same test-side kernels take any k x m sketch, so the
  GPU errors with those sketches must match the oracle's, and the tensor
  sketch must give the lower test error (Eq. 4.1) on a stream whose
  matrices share a column space.
* The training fraction (Section 4, Fig. 2): the sketch trained on the first
  D' matrices of a stream, with the mode-1 Gram accumulated chunk by chunk as
  the matrices arrive (Eq. 3.2 is a sum over d), against the oracle's Gram
  of the same D' matrices.
"""
import dataclasses

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


def _np(t):
    return t.detach().double().cpu().numpy()


def test_random_sketches_match_the_oracle_and_lose_to_the_tensor_sketch(tsk):
    spec = synth.scaled(synth.C2, 384, 288, 40, 12, k=20, r=10, storage="f32")
    tr = synth.stream(spec, "train")
    te = synth.stream(spec, "test")
    S_t, _, _, _ = oracle.train_sketch(list(tr.double().numpy()), spec.k)
    opt = [oracle.optimal_error(A, spec.r) for A in te.double().numpy()]
    h = tsk.Handle()
    ted = te.cuda()
    test_err = {}
    for name, S in (("tensor", torch.tensor(S_t, dtype=torch.float32)),
                    ("gauss", synth.random_sketch("gauss", spec.k, spec.m, 1)),
                    ("sign", synth.random_sketch("sign", spec.k, spec.m, 1))):
        e = _np(h.approx_batch(ted, S.cuda(), spec.r)["err"])
        ref = [oracle.scw(A, S.double().numpy(), spec.r, dense=False)["err"]
               for A in te.double().numpy()]
        assert np.max(np.abs(e - ref) / ref) <= GAP, name
        test_err[name] = oracle.test_error(e, opt)
    assert test_err["tensor"] < test_err["gauss"]
    assert test_err["tensor"] < test_err["sign"]
    h.close()


def test_training_fraction_with_a_streamed_gram(tsk):
    pool = dataclasses.replace(synth.scaled(synth.C2, 256, 192, 60, 10, k=12, r=6,
                                            storage="f32"))
    tr = synth.stream(pool, "train", device="cuda")
    h = tsk.Handle()
    G = None
    done = 0
    for want in (3, 12, 48):  # 5 %, 20 %, 80 % of the 60
        while done < want:
            c = min(want - done, 7)
            G = h.gram([tr[i] for i in range(done, done + c)], mode=1, out=G,
                       accumulate=G is not None)
            done += c
        R = oracle.gram_mode1(list(_np(tr[:want])))
        Gn = _np(G)
        d = np.sqrt(np.diag(R))
        assert np.max(np.abs(Gn - R) / (1e-5 * np.outer(d, d))) <= 1.0, want
        S, eig, st = h.sketch_from_gram(G, pool.k, prec=tsk.FP32)
        assert st == 0
        S_o, lam = oracle.leading_eigvecs(R, pool.k)
        Sg = _np(S)
        # the objective of Eq. 3.2: the captured energy of the oracle's Gram
        cap = float(np.trace(Sg @ R @ Sg.T))
        assert cap >= (1 - 1e-4) * float(np.sum(lam[:pool.k])), want
    h.close()
