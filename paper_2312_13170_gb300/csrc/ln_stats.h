// Column statistics entry points of ln_stats.cu beyond those in
// ln_internal.h.
#pragma once

#include <cuda_runtime.h>

#include "loopnest.h"

namespace ln {

// First pass only: the FP64 column means of X (n x m) and, when off_hi is not
// NULL, their split into an FP32 pair (off_hi + off_lo) for centring. The
// same partial sums, order and final reduction as the two-pass statistics, so
// the means and the pair are bit-identical to theirs. partials as for
// col_stats.
ln_status col_mean(int n, int m, const float *X, long long ldx, double *mean, float *off_hi, float *off_lo,
                   double *partials, cudaStream_t st);

}  // namespace ln
