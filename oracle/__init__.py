"""CPU FP64 oracle for the damped least-squares solve by composed sparse QR.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library and its
Python binding) may import, call or link anything in this package.  Only `tests/`,
`__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` use it.

The oracle is deliberately plain and slow: numpy arrays in float64, explicit loops
over columns and fronts, and no blocking, fusion or reordering beyond what the paper
states.  Every function names the passage of the paper it follows
(arXiv 1802.03773, "QRkit: Sparse, Composable QR Decompositions ...").

Modules
  householder  - dense Householder QR, implicit Q, compact WY, triangular solves (Sec. 2)
  structured   - damping rows, row permutation P_r, block-diagonal (Sec. 4.1),
                 horizontal concatenation (Sec. 4.2) and vertical concatenation
                 (Sec. 4.5 / Sec. 5.2) composed into one damped solve
  banded       - block-banded QR with short block-wise Householder vectors (Sec. 4.4)
  normal       - normal equations, Eq. (1), solved by Cholesky (cross-check and the
                 FP32 Cholesky comparison path)
  refine       - Bjorck augmented-system refinement of a least-squares solution
                 (not in the paper; the textbook method, Bjorck 1967)
  curvefit     - the cubic B-spline curve-fit model used by the LM workloads
  lm           - Levenberg-Marquardt step with the Nielsen damping rule (Sec. 2, Sec. 5.2)
  mlp          - the small damping-prediction MLP: forward, backward, Adam (not in the paper)
  more         - More's two-factorization LM step: J = QR, then [R; lambda^(1/2) D] = Q'R'
                 (Sec. 5.2, Eq. LMTwoStep)
  reorder      - row and column permutations that expose a banded structure (Sec. 4.3)

Parity status of each function is stated in its module header; a function with no
independent pin says "parity unpinned".
"""
