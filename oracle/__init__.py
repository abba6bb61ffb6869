"""FP64 CPU oracle for the tensor-based sketching method (arXiv 2209.14637).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the package's
smoke check (__graft_entry__.smoke) and the CPU-baseline leg of bench.py may
import anything from here.  The CUDA library never links or calls it, and it
shares no code with the CUDA path: the only thing both sides use is the
seeded input generator in ``synth``.

Every function is a plain, slow, readable restatement of the paper in
float64 numpy, following the order and notation of the paper:

* tensor_sketch: mode-1 Gram of the training tensor and its leading
  eigenvectors, i.e. the Tucker1 sketch S* (Section 3.1, Eqs. 3.1-3.3,
  Algorithm 2), and the mode-2 analogue for the second sketch W of the
  two-sided variant (Eq. 3.6).
* scw: the SCW sketch-and-solve step (Algorithm 1) in the QR form that the
  paper allows in Section 3.2, the literal thin-SVD form, the Eckart-Young
  optimum (Section 1) and the test error (Eq. 4.1).
* refiner: the IVY training loss (Eq. 2.1) of a dense sketch and its
  analytic gradient, used by the learned sketch refiner.
* two_sided: two-sided SCW (Algorithm 3) and HOOI (Algorithm 5).
* fp8: E4M3 copies of training matrices with per-row, per-group-of-eight
  power-of-two scales, from the format's definition (the FP8 training Gram).

Library primitives (matmul, numpy.linalg.qr/svd/eigh) serve as single steps;
nothing is blocked, fused or reordered beyond what the paper states.  How
each function is pinned to something other than itself is listed in the
tests (tests/test_oracle_*.py).
"""
from .tensor_sketch import (gram_mode1, gram_mode2, leading_eigvecs,
                            canonical_signs, train_sketch)
from .scw import scw, scw_svd_form, optimal_error, test_error, scw_batch
from .refiner import ivy_loss, ivy_grad, scw_forward_parts
from .two_sided import two_sided_scw, hooi
from .fp8 import (e4m3_decode, e4m3_encode, row_scale, quantize_e4m3,
                  dequantize_e4m3)

__all__ = [
    "gram_mode1", "gram_mode2", "leading_eigvecs", "canonical_signs",
    "train_sketch", "scw", "scw_svd_form", "optimal_error", "test_error",
    "scw_batch", "ivy_loss", "ivy_grad", "scw_forward_parts",
    "two_sided_scw", "hooi", "e4m3_decode", "e4m3_encode", "row_scale",
    "quantize_e4m3", "dequantize_e4m3",
]
