// Mixed-precision solve path.
#include "hm_mixed.h"

hm_status hm_mixed_prepare(hm_ctx*) { return HM_OK; }
hm_status hm_mixed_solve(hm_ctx*, hm::cplx*, const hm::cplx*, int) { return HM_ERR_STATE; }
hm_status hm_mixed_apply(hm_ctx*, int, hm::cplx*, const hm::cplx*, int) { return HM_ERR_STATE; }
void hm_mixed_release(hm_ctx*) {}
