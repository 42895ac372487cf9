"""FP64 CPU oracle for the GLS map-making solver of Szydlarski, Grigori & Stompor,
"Accelerating the cosmic microwave background map-making procedure through
preconditioning" (arXiv 1408.3048).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct restatement
of what the paper computes, used to check the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline / reference arm) may
import it.  It shares no code with the CUDA path (``paper_1408_3048_gb300``) and
imports nothing from it; both take their inputs from the seeded generators in
``paper_1408_3048_gb300.synth``, which hold none of the method's arithmetic.

Everything is float64 NumPy / SciPy.  Library primitives used as single steps:
``np.convolve`` (direct convolution), ``np.fft`` / ``scipy.signal.fftconvolve``
(a second, FFT route for the Toeplitz product), ``np.linalg`` (dense solves,
eigenvalues), ``scipy.linalg.lu_factor`` (LU of the coarse operator).

Modules
-------
noise     Eq. 19 noise PSD -> inverse-PSD Toeplitz row, Eq. 28 apodisation window,
          positive-definiteness of the banded symbol (Sec. 2.1, App. D).
pointing  Observed-pixel set, hit counts, P x (de-pointing) and P^T y (pointing),
          Eq. 1-2 and the full-column-rank restriction of Sec. 2.
toeplitz  Block-diagonal banded Toeplitz N^-1 (Eq. 4, band of Sec. 4.1.4) applied
          by direct convolution, by a dense matrix (tiny) and by FFT.
system    A x = P^T N^-1 P x (Eq. 5, 8), b = P^T N^-1 d (Eq. 7), dense A (tiny).
precond   M_BD (Eq. 10); deflation R (Eq. 11); M_2lvl (Eq. 12, App. C);
          a-posteriori coarse space from CG-Lanczos Ritz pairs (Sec. 3.3.2, App. A).
pcg       Preconditioned CG (Sec. 3.1) with the stopping rule of Sec. 5.1; dense
          Cholesky GLS solve (Eq. 3) for tiny problems.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against a closed form, an invariant, a brute-force or
dense computation, or a second independent route.
"""
