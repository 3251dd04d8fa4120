"""ORACLE -- test infrastructure only.

A plain, slow, FP64 CPU statement of what the accelerated path computes, written from the paper
(arXiv 2312.00538, Wagner, Pearson, Stoll) and, where the paper is silent, from the readings listed
in the repository's design notes. It shares no code, headers, tables or constants with the CUDA
library, and it does not import it. Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import, call or execute anything in this package; the library itself never
falls back to it.

Modules:
  kernel   direct ANOVA-kernel matvec (C, OpenMP) and the dense kernel matrix (Sec. 3).
  nfft     trigonometric-polynomial kernel approximation, direct NDFTs and a plain NFFT
           fast summation (Sec. 3, fast-summation factorisation).
  ipm      Algorithm 1 with dense Newton solves (Sec. 2, eq. (Newton)).
  precond  Algorithm 2 (pivoted Cholesky), Nystrom, Woodbury and the saddle preconditioner
           (Secs. 4-5).
  minres   preconditioned MINRES (Paige and Saunders), the Krylov method named in Sec. 3 and 5.
"""
