// Native H-matrix build and GPU scaling (filled in below).
#include "hm_internal.h"

extern "C" {
hm_status hm_build(const double*, int, const int*, int, const hm_params*, hm_handle*) {
  return HM_ERR_STATE;
}
hm_status hm_compute_scaling(hm_handle h) { return h ? HM_ERR_STATE : HM_ERR_INVALID; }
hm_status hm_plane_wave_rhs(hm_handle h, const double*, const double*, const int*, int, void*) {
  return h ? HM_ERR_STATE : HM_ERR_INVALID;
}
}
