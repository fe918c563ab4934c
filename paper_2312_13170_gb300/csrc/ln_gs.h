// Host-side launchers of the Gram-Schmidt QR (ln_gs.cu), called by
// ln_gramschmidt after validation. Q (m x n, ldq) already holds a copy of A
// and is factorised in place; R is n x n (ldr). Both device pointers.
#pragma once

#include <cuda_runtime.h>

#include "loopnest.h"

namespace ln {

// Plain form: the benchmark's three kernels per column (norm, scale, project).
ln_status gs_plain(int m, int n, float *Q, long long ldq, float *R, long long ldr, cudaStream_t st);

// Internalized form: blocked modified Gram-Schmidt, one CTA per 32-column
// panel plus a trailing-update kernel per panel.
ln_status gs_blocked(int m, int n, float *Q, long long ldq, float *R, long long ldr, cudaStream_t st);

// Tuning: rows per thread of the register-resident panel kernel (2 or 4).
int tune_gs_rows();

}  // namespace ln
