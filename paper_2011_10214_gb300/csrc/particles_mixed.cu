// MIXED-precision particle cycle and FP32/FP64-refined PCG (in progress):
// until these kernels land, contexts created with PIFEPIC_MIXED report
// cudaErrorNotSupported from every mixed launcher.
#include "internal.h"

namespace pf {
cudaError_t set_mixed_tables(const TetTables&) { return cudaSuccess; }
cudaError_t build_pcg_graph_mixed(Ctx&) { return cudaErrorNotSupported; }
cudaError_t launch_pcg_mixed(Ctx&) { return cudaErrorNotSupported; }
cudaError_t launch_flatten_mixed_to_f64(Ctx&, int, PArr, unsigned long long*) { return cudaErrorNotSupported; }
cudaError_t launch_build_bins_mixed(Ctx&, int, PArr, long long, bool) { return cudaErrorNotSupported; }
cudaError_t launch_push_mixed(Ctx&) { return cudaErrorNotSupported; }
cudaError_t launch_movers_mixed(Ctx&) { return cudaErrorNotSupported; }
cudaError_t launch_inject_mixed(Ctx&) { return cudaErrorNotSupported; }
cudaError_t launch_rebin_mixed(Ctx&) { return cudaErrorNotSupported; }
cudaError_t launch_deposit_all_mixed(Ctx&) { return cudaErrorNotSupported; }
cudaError_t launch_half_kick_mixed(Ctx&) { return cudaErrorNotSupported; }
}  // namespace pf
