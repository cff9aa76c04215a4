// Mixed-precision path (low-precision alpha / far factors, FP64 D^-1 and
// FP64 refinement).  Implemented in hm_mixed.cu.
#pragma once
#include "hm_internal.h"

hm_status hm_mixed_prepare(hm_ctx* h);
hm_status hm_mixed_solve(hm_ctx* h, hm::cplx* X, const hm::cplx* B, int nrhs);
hm_status hm_mixed_apply(hm_ctx* h, int op, hm::cplx* Y, const hm::cplx* X, int nrhs);
void hm_mixed_release(hm_ctx* h);

namespace hm {
// the complex64 copies of alpha, T_G and the far factors: rebuilt from the
// host copies when they were dropped (for CUDA-core launches and new tiles),
// or dropped once every tensor-core list has its tiles
hm_status mixed_ensure_c64(hm_ctx* h);
void mixed_drop_c64(hm_ctx* h);
}
