"""Seeded synthetic data streams shaped like the paper's workloads.

This module only draws inputs.  It holds none of the method's arithmetic (no
Gram, no eigensolver, no sketch, no SCW): both the FP64 oracle and the CUDA
path consume what it produces, and neither is imported here.

The paper's datasets (HSI 1024x768, Logo 3240x1920, MRI 217x181; Section 4,
Table 1) are not available, so every stream is the "drifting shared subspace"
model below, which keeps the property the method relies on: all matrices of
a stream share most of their leading column space (Section 1, "strong
relevance among matrices").

    A_d = orth(U0 + delta * E_d) @ diag(sigma) @ G_d + nu * N_d

U0 (m x L) is orth(Gaussian) drawn from the stream seed; E_d (m x L),
G_d (L x n) and N_d (m x n) are i.i.d. N(0, 1) drawn from a per-matrix seed,
so any matrix of a stream can be regenerated on its own and in any order.
orth() is a Householder QR with the signs fixed so that diag(R) >= 0.

Draws use torch generators on the requested device, so a GPU run can make
the multi-gigabyte streams in seconds; the same call on the CPU gives a
different (but equally seeded) stream.  Tests that compare the two paths
therefore generate once and hand the same tensors to both sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

BASE_SEED = 20220929


@dataclass(frozen=True)
class StreamSpec:
    """One synthetic stream: sizes, spectrum and the method's k, r."""
    name: str
    m: int
    n: int
    n_train: int
    n_test: int
    k: int
    r: int
    latent: int
    sigma: tuple
    delta: float
    nu: float
    storage: str          # "f64", "f32" or "bf16": element type of A in HBM
    seed: int

    @property
    def torch_dtype(self):
        return {"f64": torch.float64, "f32": torch.float32,
                "bf16": torch.bfloat16}[self.storage]


def _power_spectrum(L: int, p: float) -> tuple:
    return tuple(float(i) ** (-p) for i in range(1, L + 1))


def _geometric_spectrum(L: int, q: float) -> tuple:
    return tuple(q ** i for i in range(L))


# The five workloads.  C1 is the FP64 correctness case, C2 takes HSI's shape
# with the paper's k=20, r=10 (Section 4), C3 is the 2048x2048 BF16 precision
# case, C5 is the learned-refiner case (HSI shape again).  The ragged batch
# (C4) is built by ragged_batch() below.
C1 = StreamSpec("c1_fp64_128x96", 128, 96, 50, 20, 10, 5, 32,
                _geometric_spectrum(32, 0.8), 0.05, 0.01, "f64", BASE_SEED + 1)
C2 = StreamSpec("c2_fp32_1024x768", 1024, 768, 400, 200, 20, 10, 64,
                _power_spectrum(64, 1.2), 0.05, 1e-3, "f32", BASE_SEED + 2)
C3 = StreamSpec("c3_bf16_2048x2048", 2048, 2048, 1000, 500, 40, 20, 80,
                _power_spectrum(80, 1.2), 0.05, 1e-3, "bf16", BASE_SEED + 3)
C5 = StreamSpec("c5_refiner_1024x768", 1024, 768, 400, 200, 20, 10, 64,
                _power_spectrum(64, 1.2), 0.05, 1e-3, "f32", BASE_SEED + 5)
SPECS = {s.name: s for s in (C1, C2, C3, C5)}


def scaled(spec: StreamSpec, m: int, n: int, n_train: int, n_test: int,
           k: Optional[int] = None, r: Optional[int] = None,
           storage: Optional[str] = None, name: Optional[str] = None
           ) -> StreamSpec:
    """A smaller stream with the same spectrum model (for fast tests)."""
    k = spec.k if k is None else k
    r = spec.r if r is None else r
    L = min(spec.latent, m, n)
    return StreamSpec(name or f"{spec.name}_scaled_{m}x{n}", m, n, n_train,
                      n_test, k, r, L, spec.sigma[:L], spec.delta, spec.nu,
                      storage or spec.storage, spec.seed)


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) % (2 ** 63 - 1))
    return g


def orth(M: torch.Tensor) -> torch.Tensor:
    """Orthonormal basis of the columns of M, signs fixed so diag(R) >= 0.

    The QR runs on the host (LAPACK) whatever M's device, and the result
    goes back to M's device: the tall m x L factors are small, and the
    device QR would need torch's separate CUDA linear-algebra library, which
    some profiling set-ups cannot load.
    """
    Q, R = torch.linalg.qr(M.detach().to("cpu", torch.float64))
    s = torch.sign(torch.diagonal(R, dim1=-2, dim2=-1))
    s = torch.where(s == 0, torch.ones_like(s), s)
    return (Q * s.unsqueeze(-2)).to(M.device, M.dtype)


def shared_basis(spec: StreamSpec, device="cpu", stream_id: int = 0
                 ) -> torch.Tensor:
    """U0: the stream's shared m x L orthonormal basis (FP64)."""
    g = _gen(spec.seed * 7919 + 17 + 104729 * stream_id, device)
    return orth(torch.randn(spec.m, spec.latent, generator=g, device=device,
                            dtype=torch.float64))


def stream_matrix(spec: StreamSpec, U0: torch.Tensor, d: int,
                  stream_id: int = 0) -> torch.Tensor:
    """A_d (FP64, m x n) of the stream; d indexes training then test."""
    dev = U0.device
    g = _gen((spec.seed * 1000003 + d) * 31 + stream_id * 2654435761, dev)
    m, n, L = spec.m, spec.n, spec.latent
    E = torch.randn(m, L, generator=g, device=dev, dtype=torch.float64)
    G = torch.randn(L, n, generator=g, device=dev, dtype=torch.float64)
    N = torch.randn(m, n, generator=g, device=dev, dtype=torch.float64)
    sig = torch.tensor(spec.sigma[:L], device=dev, dtype=torch.float64)
    U = orth(U0 + spec.delta * E)
    return (U * sig) @ G + spec.nu * N


def stream(spec: StreamSpec, which: str = "test", device="cpu",
           count: Optional[int] = None, start: int = 0,
           dtype: Optional[torch.dtype] = None) -> torch.Tensor:
    """A stacked block of stream matrices, shape (count, m, n).

    which="train" indexes d in [0, n_train); which="test" indexes
    d in [n_train, n_train + n_test).  The result is cast to the spec's
    storage type unless dtype is given.
    """
    total = spec.n_train if which == "train" else spec.n_test
    base = 0 if which == "train" else spec.n_train
    count = total - start if count is None else count
    dtype = spec.torch_dtype if dtype is None else dtype
    U0 = shared_basis(spec, device)
    out = torch.empty(count, spec.m, spec.n, dtype=dtype, device=device)
    for i in range(count):
        out[i] = stream_matrix(spec, U0, base + start + i).to(dtype)
    return out


@dataclass
class RaggedItem:
    m: int
    n: int
    k: int
    r: int
    spec: StreamSpec = field(repr=False)


def ragged_sizes(count: int = 512, seed: int = BASE_SEED + 4,
                 m_range=(256, 4096), n_range=(256, 2048),
                 ks: Sequence[int] = (10, 20, 40)) -> List[RaggedItem]:
    """Sizes of the ragged batch: m, n log-uniform, k uniform over ks, r=k/2.

    Each item is its own small stream (latent rank 2k, sigma_i = i^-1.2,
    drift 0.05, noise 1e-3, 8 training draws); item_sketch() draws the
    sketch it is approximated with.  Sizes are not rounded: most rows of a
    contiguous BF16 item do not start on a 16-byte boundary.
    """
    rng = np.random.default_rng(seed)
    items = []
    for i in range(count):
        m = int(round(math.exp(rng.uniform(math.log(m_range[0]),
                                           math.log(m_range[1])))))
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]),
                                           math.log(n_range[1])))))
        k = int(ks[rng.integers(0, len(ks))])
        k = min(k, m, n)
        L = min(2 * k, m, n)
        spec = StreamSpec(f"ragged_{i}", m, n, 8, 1, k, max(1, k // 2), L,
                          _power_spectrum(L, 1.2), 0.05, 1e-3, "bf16",
                          seed * 1009 + i)
        items.append(RaggedItem(m, n, k, max(1, k // 2), spec))
    return items


def item_sketch(item: RaggedItem, device="cpu", spread: float = 0.1,
                dtype=torch.float32) -> torch.Tensor:
    """A k x m row-orthonormal sketch for one ragged item: the first k
    directions of the item's shared basis U0, each perturbed by a Gaussian
    vector of norm about `spread`, orthonormalised.  It stands in for a
    sketch trained on the item's own stream (a trained sketch lies near the
    same leading subspace) and is an input to both the oracle and the GPU."""
    spec = item.spec
    U0 = shared_basis(spec, "cpu")
    g = _gen(spec.seed * 6151 + 3, "cpu")
    E = torch.randn(spec.m, item.k, generator=g, dtype=torch.float64)
    Sm = orth(U0[:, :item.k] + (spread / math.sqrt(spec.m)) * E)
    return Sm.T.contiguous().to(device, dtype)


def random_sketch(kind: str, k: int, m: int, seed: int, device="cpu",
                  dtype=torch.float32) -> torch.Tensor:
    """The data-oblivious sketches of classical SCW (Section 1): a k x m
    Gaussian matrix with N(0, 1/k) entries, or a sign (Rademacher) matrix
    with entries +-1/sqrt(k)."""
    g = _gen(seed * 7 + (1 if kind == "gauss" else 2), "cpu")
    if kind == "gauss":
        S = torch.randn(k, m, generator=g, dtype=torch.float64) / math.sqrt(k)
    elif kind == "sign":
        b = torch.randint(0, 2, (k, m), generator=g, dtype=torch.int64)
        S = (2.0 * b.to(torch.float64) - 1.0) / math.sqrt(k)
    else:
        raise ValueError(f"unknown sketch kind {kind!r}")
    return S.to(device, dtype).contiguous()


def ragged_batch(items: Sequence[RaggedItem], device="cpu", pad_rows: bool = False,
                 d: int = 8) -> List[torch.Tensor]:
    """The test matrix (index d: after the 8 training draws) of every item,
    BF16.  With pad_rows the rows are laid out with a leading dimension
    rounded up to 8 elements (16 bytes), the storage a producer chooses
    for the tensor-core path; the matrices keep their n columns (views)."""
    out = []
    for it in items:
        U0 = shared_basis(it.spec, device)
        A = stream_matrix(it.spec, U0, d).to(torch.bfloat16)
        if pad_rows:
            ld = (it.n + 7) // 8 * 8
            buf = torch.zeros(it.m, ld, dtype=torch.bfloat16, device=device)
            buf[:, :it.n] = A
            A = buf[:, :it.n]
        out.append(A)
    return out
