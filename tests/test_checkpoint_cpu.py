"""Checkpoint files on the host (no GPU): the array file for S, W and dS, and
the learned refiner's resumable state.

The byte layout is pinned independently of the library: the expected files
are packed here with Python's struct module (little-endian) from the format
that include/tsk.h documents, and the library's files must equal them byte
for byte.  Round trips, and rejection of malformed or short files, go through
the C ABI.
"""
import ctypes as C
import os
import struct

import numpy as np
import pytest
import torch

import paper_2209_14637_gb300 as tsk


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(tsk.LIB_PATH):
        from paper_2209_14637_gb300 import build
        build.build()
    return tsk.load_library()


def _array_bytes(prec, a):
    """The documented array file: magic, int32 precision, int32 0, int64 rows,
    int64 cols, then the elements row-major, little-endian."""
    rows, cols = a.shape
    hdr = struct.pack("<8siiqq", b"TSKARR1\0", prec, 0, rows, cols)
    return hdr + a.tobytes()


@pytest.mark.parametrize("dtype,prec,npt", [(torch.float64, 0, "<f8"),
                                            (torch.float32, 1, "<f4")])
def test_array_file_layout(lib, tmp_path, dtype, prec, npt):
    t = torch.arange(15, dtype=torch.float64).reshape(3, 5).to(dtype) / 7 - 1
    p = tmp_path / "s.tsk"
    tsk.save_array(str(p), t)
    want = _array_bytes(prec, t.numpy().astype(npt))
    assert p.read_bytes() == want
    assert not (tmp_path / "s.tsk.tmp").exists()


def test_bf16_array_file_holds_the_raw_bits(lib, tmp_path):
    t = torch.tensor([[1.0, -2.5, 0.15625], [3e-3, 65280.0, -0.0]], dtype=torch.bfloat16)
    p = tmp_path / "b.tsk"
    tsk.save_array(str(p), t)
    bits = t.view(torch.int16).numpy().astype("<i2")
    assert p.read_bytes() == struct.pack("<8siiqq", b"TSKARR1\0", 2, 0, 2, 3) + bits.tobytes()
    u = tsk.load_array(str(p))
    assert u.dtype == torch.bfloat16 and torch.equal(u.view(torch.int16), t.view(torch.int16))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(40, 2048), (1, 1), (0, 7)])
def test_array_round_trip(lib, tmp_path, dtype, shape):
    g = torch.Generator().manual_seed(shape[0] * 31 + shape[1])
    t = torch.randn(shape, generator=g, dtype=torch.float64).to(dtype)
    p = str(tmp_path / "a.tsk")
    tsk.save_array(p, t)
    u = tsk.load_array(p)
    assert u.dtype == dtype and tuple(u.shape) == shape
    assert torch.equal(u, t)


def test_array_load_rejects_bad_files(lib, tmp_path):
    good = _array_bytes(0, np.ones((4, 4), "<f8"))
    cases = {
        "magic": b"TSKARR2\0" + good[8:],
        "precision": good[:8] + struct.pack("<i", 9) + good[12:],
        "short": good[:-8],
        "header": good[:20],
    }
    for name, data in cases.items():
        p = tmp_path / f"{name}.tsk"
        p.write_bytes(data)
        with pytest.raises(tsk.TskError) as e:
            tsk.load_array(str(p))
        assert e.value.status == 1, name
    with pytest.raises(tsk.TskError):
        tsk.load_array(str(tmp_path / "missing.tsk"))
    # a capacity below rows x cols x element size is refused
    p = tmp_path / "ok.tsk"
    p.write_bytes(good)
    buf = (C.c_double * 15)()
    pr, r, c = C.c_int32(), C.c_int64(), C.c_int64()
    st = lib.tsk_array_load(os.fsencode(str(p)), buf, 15 * 8, C.byref(pr), C.byref(r),
                            C.byref(c))
    assert st == 1 and (r.value, c.value) == (4, 4)


def test_array_save_rejects_bad_arguments(lib, tmp_path):
    x = (C.c_double * 4)()
    p = os.fsencode(str(tmp_path / "x.tsk"))
    assert lib.tsk_array_save(p, x, 5, 2, 2) == 1       # unknown precision
    assert lib.tsk_array_save(p, x, 0, -1, 2) == 1      # negative shape
    assert lib.tsk_array_save(p, None, 0, 2, 2) == 1    # no data
    assert lib.tsk_array_save(None, x, 0, 2, 2) == 1
    assert lib.tsk_array_save(os.fsencode(str(tmp_path / "no" / "dir.tsk")), x, 0, 2, 2) == 1


def _refine_bytes(prec, step, best_loss, lr, seed, steps, batch, every, order_given, dS, best):
    k, m = dS.shape
    hdr = struct.pack("<8siiqqddQiiii", b"TSKREF1\0", prec, step, k, m, best_loss, lr, seed,
                      steps, batch, every, order_given)
    assert len(hdr) == 72
    return hdr + dS.tobytes() + best.tobytes()


@pytest.mark.parametrize("dtype,prec,npt", [(torch.float64, 0, "<f8"),
                                            (torch.float32, 1, "<f4")])
def test_refine_checkpoint_layout_and_round_trip(lib, tmp_path, dtype, prec, npt):
    g = torch.Generator().manual_seed(prec)
    dS = torch.randn(6, 40, generator=g, dtype=torch.float64).to(dtype)
    best = torch.randn(6, 40, generator=g, dtype=torch.float64).to(dtype)
    state = tsk.RefineState(best, step=1200, best_loss=0.0393125)
    p = tmp_path / "run.ckpt"
    tsk.save_refine_checkpoint(str(p), dS, state, steps=2000, batch=16, lr=1e-3,
                               eval_every=100, seed=20220929, order=None)
    want = _refine_bytes(prec, 1200, 0.0393125, 1e-3, 20220929, 2000, 16, 100, 0,
                         dS.numpy().astype(npt), best.numpy().astype(npt))
    assert p.read_bytes() == want
    c = tsk.load_refine_checkpoint(str(p), device="cpu")
    assert torch.equal(c["dS"], dS) and torch.equal(c["state"].best, best)
    assert (c["state"].step, c["state"].best_loss) == (1200, 0.0393125)
    assert (c["steps"], c["batch"], c["lr"], c["eval_every"], c["seed"], c["order_given"]) == \
        (2000, 16, 1e-3, 100, 20220929, False)
    # a run that drew its batches from an explicit order says so
    tsk.save_refine_checkpoint(str(p), dS, state, steps=2000, order=[3, 1, 4])
    assert tsk.load_refine_checkpoint(str(p), device="cpu")["order_given"] is True


def test_refine_checkpoint_rejects_bad_state_and_files(lib, tmp_path):
    dS = torch.zeros(2, 3, dtype=torch.float64)
    p = str(tmp_path / "r.ckpt")
    with pytest.raises(tsk.TskError):   # more steps taken than the run has
        tsk.save_refine_checkpoint(p, dS, tsk.RefineState(dS.clone(), step=11), steps=10)
    with pytest.raises(ValueError):     # BF16 refiner state does not exist
        tsk.save_refine_checkpoint(p, dS.bfloat16(), tsk.RefineState(dS.clone()), steps=10)
    good = _refine_bytes(0, 5, 0.5, 1e-3, 1, 10, 4, 5, 0, np.zeros((2, 3), "<f8"),
                         np.zeros((2, 3), "<f8"))
    bad = {
        "magic": b"TSKARR1\0" + good[8:],
        "step": good[:12] + struct.pack("<i", 11) + good[16:],
        "batch": good[:60] + struct.pack("<i", 0) + good[64:],
        "short": good[:-1],
    }
    for name, data in bad.items():
        q = tmp_path / f"{name}.ckpt"
        q.write_bytes(data)
        with pytest.raises(tsk.TskError) as e:
            tsk.load_refine_checkpoint(str(q), device="cpu")
        assert e.value.status == 1, name
