// k_exchange.cu -- the exchange of a point-sharded solve by peer stores
// (bsde_set_shard_peers): the corrections c_i of this rank's block of points
// are stored into every other rank's buffer, then each of those ranks'
// arrival counter for this rank is raised to the exchange's epoch; the
// rank then waits on the device, with a time bound, until every other rank
// has raised its counter in this rank's flag array.  Section 4.2 makes the
// loop over the points parallel; this is the all-gather of its results
// without a host round trip, for GPUs that address each other's memory
// (NVLink peers of one node).
//
// Buffers are double-buffered by the parity of the epoch: a rank can be at
// most one exchange ahead of another (its next push needs the other's last
// push first), so the region it writes is never the one the other is
// reading.
//
// The wait is the only spin in the library that depends on another device:
// it gives up after wait_ns (and after a fixed number of polls, should the
// global timer stall), sets ST_TIMEOUT in the status word and returns, so the
// host reads BSDE_ERR_TIMEOUT and the context stays usable.  Once the status
// holds ST_TIMEOUT, later waits of the same solve return at once.
#include "common.cuh"

namespace {

__global__ void k_exchange_push(const double* __restrict__ mine, int i0, int count, int rank,
                                int nranks, const PeerPtrs pp, size_t region_off) {
  const int q = blockIdx.y;
  if (q == rank) return;
  double* dst = pp.c[q] + region_off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    dst[i0 + i] = mine[i0 + i];
}

__device__ __forceinline__ void store_release_sys(uint32_t* p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t load_acquire_sys(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// one thread per other rank: the block stored by k_exchange_push (an
// earlier kernel on the same stream) is visible system-wide before the
// counter is raised
__global__ void k_exchange_signal(int rank, int nranks, const PeerPtrs pp, uint32_t epoch) {
  const int q = threadIdx.x;
  if (q >= nranks || q == rank) return;
  __threadfence_system();
  store_release_sys(pp.flag[q] + rank, epoch);
}

// one thread per other rank: wait until its counter in this rank's flag
// array reaches the epoch, at most wait_ns nanoseconds
__global__ void k_exchange_wait(const uint32_t* flags, int rank, int nranks, uint32_t epoch,
                                uint64_t wait_ns, int* status) {
  const int q = threadIdx.x;
  if (q >= nranks || q == rank) return;
  if (*(volatile int*)status & ST_TIMEOUT) return;  // an earlier exchange already failed
  const uint64_t t0 = global_ns();
  // the poll cap stops the loop even if the timer stalls; a poll (a
  // system-scope load, a timer read and a sleep) takes well over 100 ns, so
  // the cap is not reached before wait_ns
  const uint64_t max_polls = wait_ns / 100 + 1000;
  for (uint64_t it = 0; it < max_polls; ++it) {
    if ((int32_t)(load_acquire_sys(flags + q) - epoch) >= 0) return;
    if (global_ns() - t0 > wait_ns) break;
    __nanosleep(1000);
  }
  atomicOr(status, ST_TIMEOUT);
}

}  // namespace

cudaError_t launch_exchange_peers(const double* mine, int i0, int count, int rank, int nranks,
                                  const PeerPtrs& pp, size_t region_off, uint32_t epoch,
                                  cudaStream_t st) {
  if (nranks < 2 || nranks > BSDE_RANKS_MAX) return cudaErrorInvalidValue;
  if (count > 0) {
    int blocks = (count + 255) / 256;
    if (blocks > 64) blocks = 64;
    k_exchange_push<<<dim3(blocks, nranks), 256, 0, st>>>(mine, i0, count, rank, nranks, pp, region_off);
  }
  k_exchange_signal<<<1, BSDE_RANKS_MAX, 0, st>>>(rank, nranks, pp, epoch);
  return cudaGetLastError();
}

cudaError_t launch_exchange_wait(const uint32_t* flags, int rank, int nranks, uint32_t epoch,
                                 double wait_ms, int* status, cudaStream_t st) {
  if (nranks < 2 || nranks > BSDE_RANKS_MAX) return cudaErrorInvalidValue;
  const uint64_t ns = (uint64_t)(wait_ms * 1e6);
  k_exchange_wait<<<1, BSDE_RANKS_MAX, 0, st>>>(flags, rank, nranks, epoch, ns, status);
  return cudaGetLastError();
}
