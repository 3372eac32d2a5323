"""Plain, slow, FP64 CPU oracle for streaming tensor-ring tracking.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check in
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  The CUDA library never calls it and shares no code with it: the two meet
only in the seeded inputs of ``synth``.

It follows Yu & Li, "Tracking Tensor Ring Decompositions of Streaming
Tensors": the TR format and unfoldings (Secs. 1-2), TR-ALS-NE (Alg. 2), the
sampled subchain (Alg. 3), STR (Alg. 4), rSTR with uniform, leverage-based and
KSRFT sketches (Alg. 5 with the schedules of Algs. 7-9), and the relative
error of the experiments (Sec. 4).  Every function is written from the
definition it cites, with library primitives (matmul, SVD, pinv, FFT) as steps
and no blocking or reordering beyond the definition.

Parity status: every function here is pinned by a CPU test against brute
force, a closed form, an identity of the paper or a library routine; none is
"parity unpinned".
"""
from . import loss, philox, stream, tr  # noqa: F401
