// Staged-source row pass instantiated for PF64.
#include "rowx.cuh"

namespace edk {

ed_status rx_launch(ed_ctx* c, const P3& p, const RxPlan& rx, const double* x, double* y, const int* emax,
                    cudaStream_t st) {
  switch (rx.ncol) {
    case 4: return rx_launch_n<PF64, 4>(c, p, rx, x, y, emax, st);
    case 8: return rx_launch_n<PF64, 8>(c, p, rx, x, y, emax, st);
    case 13: return rx_launch_n<PF64, 13>(c, p, rx, x, y, emax, st);
    default: return rx_launch_n<PF64, 27>(c, p, rx, x, y, emax, st);
  }
}

}  // namespace edk
