// Allocation-free transport sweep: the partial scalar-flux sums that rte_sweep keeps in memory
// owned by the batch live here in one fixed device array that is part of the library image.
//
// Who needs it: callers that must not allocate device memory while they run -- for example a
// host framework whose caching allocator already reserved the device's memory, or a latency-
// bound service loop where a cudaMalloc (which can synchronise the device and fragment memory)
// is not allowed.  They create and parameterise a batch once at set-up, then call this entry
// point as often as they like without the library allocating anything.
#include "common.cuh"

namespace rte {

int sweep_launch_with_scratch(rte_batch_t bt, const double* rho_in, double* rho_out,
                              int with_source, cudaStream_t st, double* partial);

// 2^21 doubles = 16 MiB of partial sums, allocated by the CUDA runtime when the library's device
// code is loaded on a GPU and held by that GPU until the process exits.
constexpr size_t kStaticScratchDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_sweep_scratch[kStaticScratchDoubles];

// Device address of the static array on the current device.  In host code the symbol name only
// stands for the array; its device address has to be looked up.  The lookup is repeated on every
// call (no cached address can outlive a device reset).  Under lazy module loading (the CUDA
// default) the first lookup on a device loads this file's device code and with it allocates the
// 16 MiB array; batch creation makes that first lookup (static_scratch_preload), so the
// allocation happens at set-up and never inside rte_sweep_static.
static int static_scratch(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_sweep_scratch);
  if (e != cudaSuccess || !p)
    return fail(e == cudaErrorMemoryAllocation ? RTE_ENOMEM : RTE_ECUDA,
                std::string("cudaGetSymbolAddress(static sweep scratch): ") + cudaGetErrorString(e));
  *out = static_cast<double*>(p);
  return RTE_OK;
}

int static_scratch_preload() {
  double* p = nullptr;
  return static_scratch(&p);
}

}  // namespace rte

using namespace rte;

extern "C" int rte_sweep_static(rte_batch_t b, const double* rho_in, double* rho_out,
                                int with_source, void* stream) {
  if (!b || !rho_in || !rho_out) return fail(RTE_EINVAL, "rte_sweep_static: null argument");
  RTE_TRY(params_ready(b, "rte_sweep_static"));
  if (rho_in == rho_out) return fail(RTE_EINVAL, "rte_sweep_static: rho_out aliases rho_in");
  if (((uintptr_t)rho_in | (uintptr_t)rho_out) & 15)
    return fail(RTE_EINVAL, "rte_sweep_static: arrays must be 16-byte aligned");
  const size_t need = (size_t)b->B * b->groups.size() * b->disc->n_dof;
  if (need > kStaticScratchDoubles)
    return fail(RTE_EINVAL, "rte_sweep_static: batch needs " + std::to_string(need) +
                                " doubles of partial sums, more than the static scratch holds (" +
                                std::to_string(kStaticScratchDoubles) + "); use rte_sweep");
  DeviceGuard g(b->disc->device);
  double* scratch = nullptr;
  RTE_TRY(static_scratch(&scratch));
  // every partial of every instance is written by the sweep before the reduction reads it, so the
  // previous call's contents never leak into this one and nothing needs clearing
  return sweep_launch_with_scratch(b, rho_in, rho_out, with_source, (cudaStream_t)stream, scratch);
}
