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
};

size_t df_operator_bytes(int64_t n);
size_t df_partials_bytes(int64_t n);  // W, wsplit and the error flag together
// Fill op.hi/op.lo from the full symmetric C (op.hi, op.W, op.wsplit set by the caller).
int df_operator_build(cudaStream_t st, int64_t n, const double *C, int64_t ldc, DfOperator &op);
// z = (C_hi + C_lo) w
int df_symv(cudaStream_t st, const DfOperator &op, const double *w, double *z);

}  // namespace gs
