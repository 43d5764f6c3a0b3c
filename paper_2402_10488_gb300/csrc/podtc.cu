// Dense POD projections on the fifth-generation tensor cores (tcgen05, BF16 operands, FP32
// accumulators in tensor memory).
//
// The online ROM steps (ROMSA, Eq. (rom_correction); ROMIG, Sec. 3.1.2) are two skinny dense
// products against a basis U of r <= 32 columns of length n:
//   project   P[b][i] = sum_e U[i][e] X[b][e]      (the reduced right-hand side of each instance)
//   lift      Y[b][e] = sum_i U[i][e] C[b][i]      (the full-space correction of each instance)
// In FP64 both run on GB300's FP64 pipe (2 r n FLOP per instance); with BF16 operands and FP32
// accumulation they are bound by reading X / writing Y in HBM instead.
//
// GB300 mapping.  One CTA of 128 threads owns one accumulator tile D (128 lanes x N columns of
// FP32) in tensor memory.  The operands are FP64 in global memory, so they are converted to BF16
// by the CTA's threads on their way into shared memory (TMA cannot convert), written in the
// canonical K-major layout without swizzle: 8 x 16-byte core matrices, LBO = 128 B between core
// matrices along K, SBO between 8-row groups.  After a proxy fence and a block barrier one thread
// issues tcgen05.mma (M = 128, K = 16 per instruction) and commits it to an mbarrier; all waits on
// an mbarrier are bounded and record a timeout in the caller's status word instead of hanging.
//   project: D = X_tile (M = 128 instances) x U^T (N = 32 basis vectors), K = a chunk of e,
//            staged 64 elements of K at a time through two shared-memory buffers so that the
//            conversion of stage s+1 overlaps the MMAs of stage s; each chunk's FP32 tile goes
//            to the workspace and a second kernel sums the chunks in a fixed order in FP64
//            (deterministic, no atomics).
//   lift:    D = U^T tile (M = 128 entries e) x C^T (N = instances, <= 256 per tile), K = r
//            padded to 32; the epilogue writes Y[b][e] with consecutive lanes on consecutive e.
#include <cuda_bf16.h>

#include "common.cuh"

namespace rte {
namespace {

constexpr int kTcThreads = 128;
constexpr int kProjK = 64;       // K elements per shared-memory stage of the projection
constexpr int kProjN = 32;       // basis vectors per projection tile (r <= 32)
constexpr int kLiftK = 32;       // r padded to the MMA's K granularity (2 x 16)
constexpr int kLiftN = 256;      // instances per lift tile (the largest N of one MMA)
constexpr long long kSpinLimit = 1ll << 26;  // polls of mbarrier.try_wait at most
constexpr uint64_t kWaitNs = 1000000000ull;   // and at most about one second of waiting

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of tcgen05: start address, leading-dimension byte offset (K
// direction), stride byte offset (M/N direction), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the completion of phase `parity` of an mbarrier: false once about kWaitNs
// nanoseconds (or kSpinLimit polls) have passed without it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (long long it = 0; it < kSpinLimit; ++it) {
    if ((it & 255) == 255 && global_ns() - t0 > kWaitNs) return false;
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// whole warp: allocate / free `ncols` tensor-memory columns (a power of two >= 32)
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// two FP64 values rounded (once, to nearest even) to BF16; `lo` at the lower address
__device__ __forceinline__ uint32_t pack_bf16x2(double lo, double hi) {
  const __nv_bfloat162 h = __halves2bfloat162(__double2bfloat16(lo), __double2bfloat16(hi));
  return *reinterpret_cast<const uint32_t*>(&h);
}

// 8 consecutive elements of row `row` from k0 (zero beyond n), as 8 BF16 in one 16-byte word
__device__ __forceinline__ uint4 load8_bf16(const double* __restrict__ rowp, int k0, int n) {
  double v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = k0 + q < n ? rowp[k0 + q] : 0.0;
  return make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                    pack_bf16x2(v[6], v[7]));
}

// Byte offset of the 16-byte core-matrix row holding (row, k .. k+7) in a K-major tile whose K
// extent is kext: core matrices along K are 128 B apart, 8-row groups kext/8 * 128 B apart.
__device__ __forceinline__ uint32_t kmajor_off(int row, int k, int kext) {
  return (uint32_t)((row >> 3) * (kext / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16);
}

struct ProjArgs {
  const double* U;  // [r][n]
  const double* X;  // [B][n]
  const uint8_t* active;
  float* ws;        // [n_chunks][m_tiles * 128][32]
  int* status;
  int r, n, B, kc;  // kc: K elements per chunk (multiple of kProjK)
};

// One (chunk, 128-instance tile) of the projection: ws[chunk][m][i] = sum over the chunk of
// U[i][e] X[m][e] with BF16 operands and FP32 accumulation in tensor memory.
__global__ void __launch_bounds__(kTcThreads) pod_project_tc_kernel(const ProjArgs A) {
  constexpr int kAbytes = 128 * kProjK * 2, kBbytes = kProjN * kProjK * 2;
  __shared__ __align__(1024) uint8_t sbuf[2][kAbytes + kBbytes];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int chunk = blockIdx.x, m0 = blockIdx.y * 128;
  const int k_begin = chunk * A.kc, k_end = min(A.n, k_begin + A.kc);
  const int stages = (k_end - k_begin + kProjK - 1) / kProjK;
  if (tid == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
  }
  if (warp == 0) tmem_alloc(&tslot, 32);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  const uint32_t idesc = idesc_bf16(128, kProjN);
  bool ok = true;
  for (int s = 0; s < stages; ++s) {
    const int buf = s & 1;
    if (s >= 2) ok = mbar_wait(&bar[buf], ((s - 2) >> 1) & 1) && ok;  // MMAs of stage s-2 done
    uint8_t* As = sbuf[buf];
    uint8_t* Bs = sbuf[buf] + kAbytes;
    const int k0 = k_begin + s * kProjK;
    // A: 128 rows x 8 groups of 8; a warp takes 32 consecutive rows of one group
    for (int g = tid; g < 128 * (kProjK / 8); g += kTcThreads) {
      const int kg = g >> 7, row = g & 127, m = m0 + row;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (m < A.B && (!A.active || A.active[m]) && k0 + kg * 8 < k_end)
        v = load8_bf16(A.X + (size_t)m * A.n, k0 + kg * 8, k_end);
      *reinterpret_cast<uint4*>(As + kmajor_off(row, kg * 8, kProjK)) = v;
    }
    for (int g = tid; g < kProjN * (kProjK / 8); g += kTcThreads) {
      const int kg = g / kProjN, row = g % kProjN;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (row < A.r && k0 + kg * 8 < k_end) v = load8_bf16(A.U + (size_t)row * A.n, k0 + kg * 8, k_end);
      *reinterpret_cast<uint4*>(Bs + kmajor_off(row, kg * 8, kProjK)) = v;
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs);
#pragma unroll
      for (int kk = 0; kk < kProjK / 16; ++kk)
        mma_bf16(tmem, smem_desc(a0 + 256 * kk, 128, (kProjK / 8) * 128),
                 smem_desc(b0 + 256 * kk, 128, (kProjK / 8) * 128), idesc, (s > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&bar[buf]);
    }
  }
  if (stages > 0) ok = mbar_wait(&bar[(stages - 1) & 1], ((stages - 1) >> 1) & 1) && ok;
  tc_fence_after();
  // epilogue: warp w holds lanes 32w..32w+31 = instances m0 + 32w + lane
  const int m = m0 + 32 * warp + lane;
  float v[32];
  tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), v);
  const int mt = gridDim.y * 128;
  float* out = A.ws + ((size_t)chunk * mt + m) * kProjN;
  if (stages == 0) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < 32; i += 4)
    *reinterpret_cast<float4*>(out + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  if (!ok && lane == 0) atomicExch(A.status, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 32);
}

// out[b][i] = sum over chunks of ws[chunk][b][i] in FP64, chunks in order
__global__ void pod_project_reduce_kernel(const float* __restrict__ ws, int n_chunks, int mt, int r,
                                          int B, const uint8_t* active, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * r) return;
  const int b = t / r, i = t % r;
  if (active && !active[b]) return;
  double s = 0.0;
  for (int c = 0; c < n_chunks; ++c) s += (double)ws[((size_t)c * mt + b) * kProjN + i];
  out[t] = s;
}

struct LiftArgs {
  const double* U;  // [r][n]
  const double* C;  // [B][r]
  const uint8_t* active;
  double* Y;        // [B][n]
  int* status;
  int r, n, B;
  int no_mma;       // injected fault (tests of the failure path): issue no MMA, so the wait runs out
};

// One (128 entries of e, <= 256 instances) tile of the lift: Y[b][e] = sum_i U[i][e] C[b][i].
__global__ void __launch_bounds__(kTcThreads) pod_lift_tc_kernel(const LiftArgs A) {
  constexpr int kAbytes = 128 * kLiftK * 2;
  extern __shared__ __align__(1024) uint8_t dsm[];
  uint8_t* As = dsm;
  uint8_t* Bs = dsm + kAbytes;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int e0 = blockIdx.x * 128, b0 = blockIdx.y * kLiftN;
  const int nb = min(kLiftN, A.B - b0);
  const int npad = (nb + 15) & ~15;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)npad) ncols <<= 1;
  if (tid == 0) mbar_init(&bar);
  if (warp == 0) tmem_alloc(&tslot, ncols);
  // A: row = e - e0, k = i; each thread one row, 8 basis vectors per 16-byte store
  {
    const int e = e0 + tid;
#pragma unroll
    for (int q = 0; q < kLiftK / 8; ++q) {
      double v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int i = 8 * q + j;
        v[j] = (i < A.r && e < A.n) ? A.U[(size_t)i * A.n + e] : 0.0;
      }
      *reinterpret_cast<uint4*>(As + kmajor_off(tid, 8 * q, kLiftK)) =
          make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                     pack_bf16x2(v[6], v[7]));
    }
  }
  // B: row = b - b0 (< npad), k = i
  for (int row = tid; row < npad; row += kTcThreads) {
    const int b = b0 + row;
    const bool use = row < nb && (!A.active || A.active[b]);
#pragma unroll
    for (int q = 0; q < kLiftK / 8; ++q) {
      double v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int i = 8 * q + j;
        v[j] = (use && i < A.r) ? A.C[(size_t)b * A.r + i] : 0.0;
      }
      *reinterpret_cast<uint4*>(Bs + kmajor_off(row, 8 * q, kLiftK)) =
          make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                     pack_bf16x2(v[6], v[7]));
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (tid == 0 && !A.no_mma) {
    const uint32_t a0 = smem_addr(As), bb0 = smem_addr(Bs), idesc = idesc_bf16(128, npad);
#pragma unroll
    for (int kk = 0; kk < kLiftK / 16; ++kk)
      mma_bf16(tmem, smem_desc(a0 + 256 * kk, 128, (kLiftK / 8) * 128),
               smem_desc(bb0 + 256 * kk, 128, (kLiftK / 8) * 128), idesc, kk > 0 ? 1u : 0u);
    mma_commit(&bar);
  }
  const bool ok = mbar_wait(&bar, 0);
  tc_fence_after();
  const int e = e0 + 32 * warp + lane;
  for (int c0 = 0; c0 < npad; c0 += 32) {
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int row = c0 + j, b = b0 + row;
      if (row < nb && e < A.n && (!A.active || A.active[b])) A.Y[(size_t)b * A.n + e] = (double)v[j];
    }
  }
  if (!ok && lane == 0) atomicExch(A.status, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, ncols);
}

constexpr size_t kLiftSmem = 128 * kLiftK * 2 + kLiftN * kLiftK * 2;
// dynamic shared memory requested per lift CTA: at least 80 KB, so at most two lift CTAs (each
// holding up to 256 tensor-memory columns) share an SM's 512 columns
constexpr size_t kLiftSmemReq = kLiftSmem > 80 * 1024 ? kLiftSmem : 80 * 1024;

}  // namespace

// ---- host side -------------------------------------------------------------------------------

// one-shot injected fault of the tensor-core products (rte_fault_inject)
static std::atomic<int> g_fault{0};

// Chunking of the projection's K range: about two CTAs per SM over all instance tiles.
static void proj_chunks(int n, int B, int n_sm, int* kc, int* n_chunks, int* mt) {
  *mt = (B + 127) / 128;
  const int want = std::max(1, (2 * n_sm + *mt - 1) / *mt);
  int k = (n + want - 1) / want;
  k = std::max(kProjK, (k + kProjK - 1) / kProjK * kProjK);
  *kc = k;
  *n_chunks = (n + k - 1) / k;
}

size_t pod_project_ws_bytes(int n, int B, int n_sm) {
  int kc, nch, mt;
  proj_chunks(n, B, n_sm, &kc, &nch, &mt);
  return sizeof(int) * 64 + sizeof(float) * (size_t)nch * mt * 128 * kProjN;
}

// The projection into `out` [B][r] (FP64); ws: pod_project_ws_bytes() bytes, its first word the
// status (set to 1 when a device-side wait gave up; the caller clears it).
int pod_project_bf16(const double* U, int r, int n, const double* X, int B, const uint8_t* active,
                     double* out, void* ws, int n_sm, cudaStream_t st) {
  if (r < 1 || r > kProjN || n < 1 || B < 1) return fail(RTE_EINVAL, "BF16 projection: bad sizes");
  int kc, nch, mt;
  proj_chunks(n, B, n_sm, &kc, &nch, &mt);
  ProjArgs A{U, X, active, reinterpret_cast<float*>(static_cast<int*>(ws) + 64), static_cast<int*>(ws),
             r, n, B, kc};
  pod_project_tc_kernel<<<dim3(nch, mt), kTcThreads, 0, st>>>(A); RTE_NOTE_LAUNCH();
  pod_project_reduce_kernel<<<(B * r + 255) / 256, 256, 0, st>>>(A.ws, nch, mt * 128, r, B, active,
                                                                  out); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

// The lift into Y [B][n] (FP64; rows of inactive instances untouched); status: device int set to 1
// when a device-side wait gave up.
int pod_lift_bf16(const double* U, int r, int n, const double* C, int B, const uint8_t* active,
                  double* Y, int* status, cudaStream_t st) {
  if (r < 1 || r > kLiftK || n < 1 || B < 1) return fail(RTE_EINVAL, "BF16 lift: bad sizes");
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    RTE_CUDA_TRY(cudaFuncSetAttribute(pod_lift_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kLiftSmemReq));
    attr_set[dev] = true;
  }
  LiftArgs A{U, C, active, Y, status, r, n, B, g_fault.exchange(0) == RTE_FAULT_LIFT_NO_MMA ? 1 : 0};
  pod_lift_tc_kernel<<<dim3((n + 127) / 128, (B + kLiftN - 1) / kLiftN), kTcThreads, kLiftSmemReq,
                       st>>>(A); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

}  // namespace rte

using namespace rte;

static int sm_count() {
  int dev = 0, n = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

extern "C" int rte_fault_inject(int what) {
  if (what != 0 && what != RTE_FAULT_LIFT_NO_MMA) return fail(RTE_EINVAL, "rte_fault_inject: unknown fault");
  g_fault.store(what);
  return RTE_OK;
}

extern "C" int rte_pod_workspace_bytes(int r, int n, int B, int64_t* bytes) {
  if (!bytes || r < 1 || r > 32 || n < 1 || B < 1)
    return fail(RTE_EINVAL, "rte_pod_workspace_bytes: bad arguments");
  *bytes = (int64_t)pod_project_ws_bytes(n, B, sm_count());
  return RTE_OK;
}

extern "C" int rte_pod_project_bf16(const double* U, int r, int n, const double* X, int B,
                                    const uint8_t* active, double* out, void* work, void* stream) {
  if (!U || !X || !out || !work) return fail(RTE_EINVAL, "rte_pod_project_bf16: null argument");
  if (((uintptr_t)work) & 15) return fail(RTE_EINVAL, "rte_pod_project_bf16: work not 16-byte aligned");
  return pod_project_bf16(U, r, n, X, B, active, out, work, sm_count(), (cudaStream_t)stream);
}

extern "C" int rte_pod_lift_bf16(const double* U, int r, int n, const double* C, int B,
                                 const uint8_t* active, double* Y, void* work, void* stream) {
  if (!U || !C || !Y || !work) return fail(RTE_EINVAL, "rte_pod_lift_bf16: null argument");
  return pod_lift_bf16(U, r, n, C, B, active, Y, static_cast<int*>(work), (cudaStream_t)stream);
}
