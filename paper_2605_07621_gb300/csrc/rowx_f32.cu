// Staged-source row pass instantiated for PF32.
#include "rowx.cuh"

namespace edk {

ed_status rx_launch(ed_ctx* c, const P3& p, const RxPlan& rx, const float* x, float* y, const int* emax,
                    cudaStream_t st) {
  switch (rx.ncol) {
    case 4: return rx_launch_n<PF32, 4>(c, p, rx, x, y, emax, st);
    case 8: return rx_launch_n<PF32, 8>(c, p, rx, x, y, emax, st);
    default: return rx_launch_n<PF32, 13>(c, p, rx, x, y, emax, st);  // plans stop at 13 for 4-byte types
  }
}

}  // namespace edk
