// Reduced-precision composition (NV_TF32_REFINE): placeholder until the
// tensor-core scan lands.
#include "internal.h"

nv_status launch_scan_refine(nv_maps*, const double*, double*, double*, cudaStream_t) {
  return nv_fail(NV_ENOTSUP, "TF32 scan composition is not built yet");
}
