"""The seeded input generator: determinism, shapes and the stream model."""
import numpy as np
import torch

import synth


def test_orth_signs_and_orthonormality():
    g = torch.Generator().manual_seed(0)
    M = torch.randn(30, 7, generator=g, dtype=torch.float64)
    Q = synth.orth(M)
    assert torch.allclose(Q.T @ Q, torch.eye(7, dtype=torch.float64), atol=1e-13)
    R = Q.T @ M
    assert bool((torch.diagonal(R) > 0).all())
    assert torch.allclose(torch.triu(R), R, atol=1e-12)


def test_stream_is_deterministic_and_matrix_addressable():
    spec = synth.scaled(synth.C2, 64, 48, 4, 3, k=6, r=3)
    a = synth.stream(spec, "test", dtype=torch.float64)
    b = synth.stream(spec, "test", dtype=torch.float64)
    assert torch.equal(a, b)
    c = synth.stream(spec, "test", dtype=torch.float64, start=1, count=1)
    assert torch.equal(a[1], c[0])
    t = synth.stream(spec, "train", dtype=torch.float64)
    assert t.shape == (4, 64, 48)
    assert not torch.equal(t[0], a[0])


def test_stream_shares_a_column_space():
    # The span of U0 captures far more of every matrix than a random basis
    # of the same size does (drift 0.05 * N(0,1) per entry of E_d).
    spec = synth.C1
    U0 = synth.shared_basis(spec)
    A = synth.stream_matrix(spec, U0, 3)
    assert A.shape == (128, 96)
    g = torch.Generator().manual_seed(1)
    R = synth.orth(torch.randn(128, spec.latent, generator=g, dtype=torch.float64))
    out_u0 = float((A - U0 @ (U0.T @ A)).norm() / A.norm())
    out_rand = float((A - R @ (R.T @ A)).norm() / A.norm())
    assert out_u0 < 0.6 and out_u0 < 0.7 * out_rand


def test_storage_types():
    assert synth.C1.torch_dtype == torch.float64
    assert synth.C2.torch_dtype == torch.float32
    assert synth.C3.torch_dtype == torch.bfloat16
    x = synth.stream(synth.scaled(synth.C3, 32, 32, 1, 1, k=4, r=2), "test")
    assert x.dtype == torch.bfloat16


def test_ragged_sizes():
    items = synth.ragged_sizes(64)
    assert len(items) == 64
    for it in items:
        assert 256 <= it.m <= 4096 and 256 <= it.n <= 2048
        assert it.k in (10, 20, 40) and it.r == it.k // 2
    assert items[0].m == synth.ragged_sizes(64)[0].m
    full = synth.ragged_sizes(512)
    ms = np.log([it.m for it in full])
    assert abs(ms.mean() - 0.5 * (np.log(256) + np.log(4096))) < 0.15
    # sizes are not rounded: most widths are not multiples of 8
    assert sum(it.n % 8 != 0 for it in full) > 256


def test_item_and_random_sketches():
    it = synth.ragged_sizes(3)[1]
    S = synth.item_sketch(it)
    assert S.shape == (it.k, it.m) and S.dtype == torch.float32
    assert torch.allclose(S.double() @ S.double().T, torch.eye(it.k, dtype=torch.float64),
                          atol=1e-5)
    assert torch.equal(S, synth.item_sketch(it))
    g = synth.random_sketch("gauss", 20, 300, 1, dtype=torch.float64)
    assert g.shape == (20, 300) and abs(float(g.pow(2).mean()) - 1 / 20) < 0.2 / 20
    s = synth.random_sketch("sign", 20, 300, 1, dtype=torch.float64)
    assert torch.allclose(s.abs(), torch.full_like(s, 20 ** -0.5))


def test_padded_ragged_batch_keeps_the_values():
    items = synth.ragged_sizes(4, m_range=(64, 96), n_range=(33, 61))
    a = synth.ragged_batch(items)
    b = synth.ragged_batch(items, pad_rows=True)
    for x, y, it in zip(a, b, items):
        assert x.shape == y.shape == (it.m, it.n)
        assert (y.stride(0) * 2) % 16 == 0
        assert torch.equal(x, y)
