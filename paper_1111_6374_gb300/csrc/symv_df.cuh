// Double-float symmetric operator for ke1 (symv_df.cu).
#pragma once

#include "common.cuh"

namespace gs {

// C's lower triangle as fp32 hi/lo tiles plus the per-call scratch.
struct DfOperator {
  int64_t n = 0, NT = 0, npad = 0;
  float *hi = nullptr, *lo = nullptr;  // df_operator_bytes(n) starting at hi
  float2 *W = nullptr;                 // NT * npad partials
  float2 *wsplit = nullptr;            // npad split input vector
  int *err = nullptr;                  // device flag: a bounded wait of the symv kernel expired
  uint32_t spin = 0;                   // poll limit of the kernel's main-loop waits (0 = the default bound)
  unsigned long long *amax = nullptr;  // device: max |entry| (bits) of the stored matrix, after the tiles
};

// Products with the stored lower triangle: the symmetric matrix it
// completes, or the lower-triangular matrix L itself, or L^T.
enum DfMode { DF_SYM = 0, DF_ROWS = 1, DF_COLS = 2 };

size_t df_operator_bytes(int64_t n);  // the tiles plus the operator's scale
size_t df_partials_bytes(int64_t n);  // W, wsplit and the error flag together
// Fill op.hi/op.lo from the lower triangle of C (trans = false) or of C^T
// (trans = true, i.e. C's upper triangle); tri = true stores a lower-
// triangular matrix (zeros above the diagonal), else the diagonal tiles
// hold the full symmetric blocks (op.hi, op.W, op.wsplit set by the caller).
int df_operator_build(cudaStream_t st, int64_t n, const double *C, int64_t ldc, DfOperator &op, bool tri = false,
                      bool trans = false);
// z = M w with M = C_hi + C_lo: symmetric (DF_SYM), or the stored lower
// triangle L (DF_ROWS) or its transpose (DF_COLS)
int df_symv(cudaStream_t st, const DfOperator &op, const double *w, double *z, int mode = DF_SYM);

}  // namespace gs
