/*
 * qc_oracle.c -- plain FP64 CPU oracle for state-vector gate application.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file; only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header or table
 * with the CUDA implementation.
 *
 * What it computes (QCLAB++, Sec. 2, Eq. (1)): applying a gate U to a state
 * phi in C^(2^n) is the matrix-vector product psi = (I_l (x) U (x) I_r) phi.
 * The oracle does not use the paper's bit-mask index generation (Alg. 1-3);
 * it walks every basis index x and, following Definition 1 (big-endian: qubit
 * q is bit n-1-q of x, i.e. it has stride 2^(n-q-1)), picks out the groups of
 * amplitudes that the gate mixes.  For a gate on k target qubits the group of
 * x (all target bits of x zero) is { x + sum_i r_i * 2^(n-q_i-1) }, r in
 * {0,1}^k, and the group is replaced by U times the group, with the row/column
 * index of U being r read as a big-endian k-bit number (q_0 is the most
 * significant bit).  For a k=1 gate this is Eq. (3); for k=2 it is the
 * 4x4 matvec of Sec. 2.3 in the index order that Eq. (1) fixes (target
 * qubits taken in the order the caller lists them).
 *
 * Controlled gates (Sec. 2.2, Sec. 2.4): the group is updated only when every
 * control qubit c of x has the requested control state; all other amplitudes
 * are left untouched.
 *
 * Arithmetic: C99 double complex, textbook complex product
 * (-fcx-limited-range).  Each iteration of the outer loop owns a disjoint
 * group, so the OpenMP loop is race-free and the result does not depend on the
 * thread count.
 *
 * Parity pins for this file live in the CPU test-suite: the n=3 index sets of
 * Figs. 2, 3 and 6, dense Kronecker products (Eq. (1)) for n <= 6, Bell/GHZ
 * states and the QFT of a basis state against a library FFT.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_MAXK 10

/* Stride of qubit q in an n-qubit register (Definition 1). */
static uint64_t orc_stride(int n, int q) { return (uint64_t)1 << (n - q - 1); }

/* Returns 0, or -1 when the arguments do not describe a valid gate. */
static int orc_check(int n, const int* qubits, int k, const int* controls, int nc) {
  if (n < 1 || n > 40 || k < 1 || k > ORC_MAXK || nc < 0 || k + nc > n) return -1;
  for (int i = 0; i < k + nc; i++) {
    int qi = i < k ? qubits[i] : controls[i - k];
    if (qi < 0 || qi >= n) return -1;
    for (int j = 0; j < i; j++) {
      int qj = j < k ? qubits[j] : controls[j - k];
      if (qi == qj) return -1;
    }
  }
  return 0;
}

/*
 * psi <- (controlled) U applied to the k target qubits `qubits` (q_0 = most
 * significant bit of U's row/column index), conditioned on each
 * controls[i] having value cstates[i].  U is 2^k x 2^k, row-major.
 */
int orc_apply_gate(int n, cplx* psi, const cplx* U, const int* qubits, int k,
                   const int* controls, const int* cstates, int nc) {
  if (orc_check(n, qubits, k, controls, nc)) return -1;
  const int64_t N = (int64_t)1 << n;
  const int dim = 1 << k;
  uint64_t tmask = 0, cmask = 0, cval = 0;
  for (int i = 0; i < k; i++) tmask |= orc_stride(n, qubits[i]);
  for (int i = 0; i < nc; i++) {
    cmask |= orc_stride(n, controls[i]);
    if (cstates[i]) cval |= orc_stride(n, controls[i]);
  }
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < N; x++) {
    if ((uint64_t)x & tmask) continue;           /* x is not the first index of its group */
    if (((uint64_t)x & cmask) != cval) continue; /* control condition not met */
    uint64_t idx[1 << ORC_MAXK];
    cplx in[1 << ORC_MAXK];
    for (int r = 0; r < dim; r++) {
      uint64_t y = (uint64_t)x;
      for (int i = 0; i < k; i++)
        if ((r >> (k - 1 - i)) & 1) y += orc_stride(n, qubits[i]);
      idx[r] = y;
      in[r] = psi[y];
    }
    for (int r = 0; r < dim; r++) {
      cplx acc = 0;
      for (int c = 0; c < dim; c++) acc += U[(size_t)r * dim + c] * in[c];
      psi[idx[r]] = acc;
    }
  }
  return 0;
}
