// k_gram_tc.cu -- the Gram matrix A = sum_i B(t_i,x_i) B(t_i,x_i)^T of the
// normal equations (eq. alphasys, Section 3.2.2), the one dense contraction
// of Algorithm 2, on the 5th-generation tensor cores of sm_103a.
//
// A is symmetric, so only the upper 128x128 tiles (I <= J) are computed.
// Each CTA owns one tile and one slice of the point dimension (split-K over
// the n points, so that the few tiles of a p ~ 400 basis still fill the
// GPU).  Operands are FP32 basis values split as b = hi + lo with hi, lo
// both TF32 (3xTF32: hi*hi + hi*lo + lo*hi, FP32 accumulation in tensor
// memory), which keeps close to FP32 accuracy on the TF32 tensor path.
//   warp 0 / lane 0 : TMA producer (cp.async.bulk.tensor, 128B swizzle)
//   warp 1 / lane 0 : MMA issuer (tcgen05.mma.cta_group::1.kind::tf32)
//   warps 0-3       : epilogue, tcgen05.ld of the 128x128 FP32 accumulator
// A 3-stage mbarrier ring overlaps loads and MMAs.  Every wait is bounded.
// A wait for work that may never be issued (the producer waiting for a stage
// the MMA issuer has not released, the issuer waiting for loads the producer
// has not started) gives up after WAIT_LIMIT polls: the kernel then sets
// ST_TIMEOUT and stops issuing.  Before it reads or frees its tensor memory
// and before it exits, the CTA waits for everything it did issue (TMA loads
// into its shared memory, committed MMAs into its tensor memory).  Issued
// work completes without any further action of the CTA, so those drain
// waits end; their bound (DRAIN_LIMIT polls, many seconds) only keeps every
// loop finite.  If even a drain wait gave up, the accumulator is not read.
// The FP32 partial tiles are summed in FP64 in split order by a second
// kernel, so the result is deterministic.
#include <cuda.h>

#include "common.cuh"

namespace {

constexpr int TILE = 128;       // M = N = 128
constexpr int KBLK = 32;        // tf32 elements per 128-byte swizzle row
constexpr int STAGES = 3;
constexpr int TILE_BYTES = TILE * KBLK * 4;  // 16 KB
constexpr int STAGE_BYTES = 4 * TILE_BYTES;  // Ahi, Alo, Bhi, Blo
constexpr uint32_t WAIT_LIMIT = 1u << 26;    // polls before giving up on unissued work
constexpr uint32_t DRAIN_LIMIT = 1u << 30;   // polls of a wait for issued work

struct GramArgs {
  int ntile_side;  // p_pad / 128
  int splits;
  int kblocks;     // n_pad / 32
  float* part;     // [tile][split][128][128]
  int* status;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// bounded wait on the phase with the given parity; false on expiry
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          uint32_t limit = WAIT_LIMIT) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row swizzle atoms 1024 bytes apart (stride byte offset), descriptor
// version 1 (bits 46-47), no base offset (stage buffers are 1024-aligned)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for SW128 K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, N = M = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TILE >> 3) << 17) |
                           ((uint32_t)(TILE >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__global__ void __launch_bounds__(128, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
              const __grid_constant__ GramArgs ga) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-align the stage ring
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* stage_mem = base;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  __shared__ int s_fail, s_issued, s_consumed, s_acc_ok;
  volatile int* fail_flag = &s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tile (I <= J) and split
  const int tile = blockIdx.x / ga.splits;
  const int split = blockIdx.x - tile * ga.splits;
  int t = tile, I = 0;
  while (t >= ga.ntile_side - I) {
    t -= ga.ntile_side - I;
    ++I;
  }
  const int J = I + t;
  const int kb0 = (int)(((long long)split * ga.kblocks) / ga.splits);
  const int kb1 = (int)(((long long)(split + 1) * ga.kblocks) / ga.splits);
  const int nk = kb1 - kb0;

  const uint32_t bar_full = smem_u32(bars), bar_empty = smem_u32(bars + STAGES),
                 bar_acc = smem_u32(bars + 2 * STAGES);
  if (tid == 0) {
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_acc, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TILE));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      if (it >= STAGES) {
        if (!mbar_wait(bar_empty + 8 * s, (uint32_t)(((it / STAGES) - 1) & 1))) {
          atomicOr(ga.status, ST_TIMEOUT);
          *fail_flag = 1;
          break;
        }
      }
      if (*fail_flag) break;
      const uint32_t dst = smem_u32(stage_mem + s * STAGE_BYTES);
      const int kx = (kb0 + it) * KBLK;
      mbar_expect_tx(bar_full + 8 * s, STAGE_BYTES);
      tma_load_2d(dst, &map_hi, kx, I * TILE, bar_full + 8 * s);
      tma_load_2d(dst + TILE_BYTES, &map_lo, kx, I * TILE, bar_full + 8 * s);
      tma_load_2d(dst + 2 * TILE_BYTES, &map_hi, kx, J * TILE, bar_full + 8 * s);
      tma_load_2d(dst + 3 * TILE_BYTES, &map_lo, kx, J * TILE, bar_full + 8 * s);
      s_issued = it + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    int issued = 0;
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      if (!mbar_wait(bar_full + 8 * s, (uint32_t)((it / STAGES) & 1))) {
        atomicOr(ga.status, ST_TIMEOUT);
        *fail_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = smem_u32(stage_mem + s * STAGE_BYTES);
      const uint32_t a_lo = a_hi + TILE_BYTES, b_hi = a_hi + 2 * TILE_BYTES,
                     b_lo = a_hi + 3 * TILE_BYTES;
#pragma unroll
      for (int kk = 0; kk < KBLK / 8; ++kk) {
        const uint32_t off = kk * 32;  // 8 tf32 = 32 bytes along K
        mma_tf32(tmem, sdesc(a_hi + off), sdesc(b_hi + off), issued);
        issued = 1;
        mma_tf32(tmem, sdesc(a_hi + off), sdesc(b_lo + off), 1);
        mma_tf32(tmem, sdesc(a_lo + off), sdesc(b_hi + off), 1);
      }
      mma_commit(bar_empty + 8 * s);  // stage free once these MMAs complete
      s_consumed = it + 1;
    }
    // always issued: arrives once every MMA issued above has completed
    // (at once when none was issued)
    mma_commit(bar_acc);
  }
  __syncthreads();
  if (tid == 0) {
    bool ok = true;
    // failure path only: drain the loads issued but never consumed
    for (int it = s_consumed; it < s_issued; ++it)
      ok = mbar_wait(bar_full + 8 * (it % STAGES), (uint32_t)((it / STAGES) & 1), DRAIN_LIMIT) && ok;
    // drain the committed MMAs: after this the accumulator is final
    ok = mbar_wait(bar_acc, 0, DRAIN_LIMIT) && ok;
    if (!ok) atomicOr(ga.status, ST_TIMEOUT);
    s_acc_ok = ok && !*fail_flag;
  }
  __syncthreads();
  // CTA-uniform: tcgen05.ld is a warp-collective instruction
  const bool ok = s_acc_ok != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = warp * 32 + lane;
  float* dst = ga.part + (((size_t)tile * ga.splits + split) * TILE + row) * TILE;
#pragma unroll
  for (int cb = 0; cb < TILE / 32; ++cb) {
    uint32_t r[32];
    if (!(ok && nk > 0)) {
      float4* d4 = reinterpret_cast<float4*>(dst + cb * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q) d4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    float4* d4 = reinterpret_cast<float4*>(dst + cb * 32);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      d4[q] = make_float4(__uint_as_float(r[4 * q + 0]), __uint_as_float(r[4 * q + 1]),
                          __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TILE));
  }
}

// A[l1][l2] = sum over splits (FP64, split order) of the partial tiles;
// diagonal tiles are read on and above their diagonal only, so A is
// exactly symmetric.
__global__ void k_gram_reduce(int p, int ntile_side, int splits, const float* __restrict__ part,
                              double* __restrict__ A) {
  const int tile = blockIdx.y;
  int t = tile, I = 0;
  while (t >= ntile_side - I) {
    t -= ntile_side - I;
    ++I;
  }
  const int J = I + t;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // 0 .. 128*128-1
  const int r = e >> 7, c = e & 127;
  if (I == J && r > c) return;
  const int l1 = I * TILE + r, l2 = J * TILE + c;
  if (l1 >= p || l2 >= p) return;
  double s = 0.0;
  for (int q = 0; q < splits; ++q) s += (double)part[(((size_t)tile * splits + q) * TILE + r) * TILE + c];
  A[(size_t)l1 * p + l2] = s;
  A[(size_t)l2 * p + l1] = s;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* map, const float* base, int n_pad, int p_pad) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)p_pad};
  const cuuint64_t strides[1] = {(cuuint64_t)n_pad * 4};
  const cuuint32_t box[2] = {KBLK, TILE};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// number of K splits: `want` when positive (at most one per K-block of 32
// points), otherwise enough to fill about one wave of the device's SMs
int gram_tc_splits(int p_pad, int n_pad, int want) {
  const int side = p_pad / TILE;
  const int tiles = side * (side + 1) / 2;
  const int kblocks = n_pad / KBLK;
  int s = want > 0 ? want : device_sm_count() / tiles;
  if (s < 1) s = 1;
  if (s > kblocks) s = kblocks;
  return s;
}

size_t gram_tc_part_bytes(int p_pad, int n_pad, int splits) {
  const int side = p_pad / TILE;
  const int tiles = side * (side + 1) / 2;
  return (size_t)tiles * splits * TILE * TILE * sizeof(float);
}

cudaError_t launch_gram_tc(const ProblemDev& P, cudaStream_t st) {
  if (P.p_pad % TILE != 0 || P.n_pad % KBLK != 0 || !P.Bhi || !P.Blo || !P.gram_part)
    return cudaErrorInvalidValue;
  CUtensorMap mh, ml;
  if (!make_map(&mh, P.Bhi, P.n_pad, P.p_pad) || !make_map(&ml, P.Blo, P.n_pad, P.p_pad))
    return cudaErrorInvalidValue;
  GramArgs ga;
  ga.ntile_side = P.p_pad / TILE;
  ga.splits = P.gram_splits > 0 ? P.gram_splits : gram_tc_splits(P.p_pad, P.n_pad, 0);
  ga.kblocks = P.n_pad / KBLK;
  ga.part = P.gram_part;
  ga.status = P.status;
  const int tiles = ga.ntile_side * (ga.ntile_side + 1) / 2;
  const size_t smem = 1024 + (size_t)STAGES * STAGE_BYTES + 64;
  cudaError_t e =
      cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gram_tc<<<tiles * ga.splits, 128, smem, st>>>(mh, ml, ga);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid(TILE * TILE / 256, tiles);
  k_gram_reduce<<<grid, 256, 0, st>>>(P.p, ga.ntile_side, ga.splits, P.gram_part, P.A);
  return cudaGetLastError();
}
