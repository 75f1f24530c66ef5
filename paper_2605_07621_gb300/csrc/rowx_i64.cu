// Staged-source row pass instantiated for PI64.
#include "rowx.cuh"

namespace edk {

ed_status rx_launch(ed_ctx* c, const P3& p, const RxPlan& rx, const long long* x, long long* y, const int* emax,
                    cudaStream_t st) {
  switch (rx.ncol) {
    case 4: return rx_launch_n<PI64, 4>(c, p, rx, x, y, emax, st);
    case 8: return rx_launch_n<PI64, 8>(c, p, rx, x, y, emax, st);
    case 13: return rx_launch_n<PI64, 13>(c, p, rx, x, y, emax, st);
    default: return rx_launch_n<PI64, 27>(c, p, rx, x, y, emax, st);
  }
}

}  // namespace edk
