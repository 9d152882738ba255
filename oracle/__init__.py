"""FP64 CPU oracle for the JL sketching path (test infrastructure only).

This package is the plain, slow, obviously-correct restatement of what the
sketching hot path computes.  It exists to check the CUDA path; it is not part
of it.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import it.  It shares no code with the CUDA library and does
not import it; the two meet only through the seeded point/matrix generators in
``paper_2302_01977_gb300.inputs``.

Modules
-------
rng        Philox4x64-10 counter-based generator and Lemire's bounded integers
           (the paper uses an unspecified LCG; the stream layout is this
           project's reading, stated in each function).
operators  SJLT (graph and block construction, Sec. 2.4.3; data structure
           R = (B+ - B-)/sqrt(alpha), Sec. 6.1), SRHT R = DHP with the
           element formula R_ij = d_i (-1)^(i . mu_j) / sqrt(d) (Sec. 2.4.2,
           the element formula of Sec. 7.2) and the Gaussian operator N(0, 1/d) (Sec. 2.4.1), formed
           densely from their definitions, with Delta-d increments (Sec. 6.2,
           Algorithm 1).
sketch     S = A R and S' = A^T R by dense FP64 products (Sec. 6.3), the
           kernel-matrix generator, a textbook fast Walsh-Hadamard transform.
kernel_grad the matrix-free kernel sketch S = K(X, X; h) R and the gradient
           of <dS, S> with respect to X and h (chain rule of the definition;
           the paper does not differentiate the sketch).
adaptive   the global adaptive loop: first sketch with d0 + Delta-d columns,
           two-pass block Gram-Schmidt projection and the Frobenius stopping
           test (Eq. (3.1) and the remark after it; Algorithm 1).

Every function is pinned by ``tests/test_oracle_*.py`` against facts the paper
and the mathematics fix (worked example of Sec. 6.1, H H^T = nI, exact nonzero
counts, E||x^T R||^2 = ||x||^2, brute force at n <= 64, numpy's own Philox).
"""
