"""FP64 CPU oracle for the sliced tensor-network contraction of random quantum
circuits (arXiv 2111.01066).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check of the
build entry point and the CPU-baseline leg of the benchmark may import it.  The
library (the C-ABI and its CUDA kernels) never calls it, and it never calls the
library: the two share no code.  The only module both sides use is `rqcgen`,
which draws the seeded circuits and holds none of the method's arithmetic.

Contents, each written from the paper's statement of the problem:

* `statevector` -- the Schroedinger algorithm (main text, section II): apply
  every gate to a 2^n state; amplitudes are read out directly.
* `tensornet`  -- the tensor-network picture (SI, figure S2 and the TN section):
  gates are rank-2 / rank-4 tensors, the initial state and the target basis are
  rank-1 tensors, contracting the network gives an amplitude; index slicing
  (main text, section II) writes the network as a sum of smaller networks with
  the sliced indices fixed.  Contracted with numpy tensordot in complex128,
  in the oracle's own greedy order.
* `xeb` -- linear cross-entropy benchmarking and the Porter-Thomas density of
  Eq. (1) of the main text.
* `sampling` -- frugal rejection sampling of one bitstring from a batch of
  correlated amplitudes (main text, section III).

Pins (tests/test_oracle_*.py): closed-form gate actions, a Kronecker-built dense
circuit matrix, a Feynman path sum over all wire values on tiny circuits,
slice-sum identities, unit norm, Porter-Thomas moments.  The FP64 results of
this package are never tuned for speed.
"""
