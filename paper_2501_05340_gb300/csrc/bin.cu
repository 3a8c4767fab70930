// Counting sort of particles into bins (collision cells or mesh elements):
// exclusive scan of the bin counts, scatter, and a per-bin ordering by id so that
// the sorted order is canonical, independent of the atomic slot assignment.
// This is the GPU counterpart of the per-step sort of particles by host element
// (Sec. 4.3), with a uniform cell grid in place of the element list.
#include "pc_internal.cuh"

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = PC_SCAN_TILE / kScanThreads;  // 8 elements per thread

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total in *total.
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
  __shared__ int wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = warp_incl_scan(v);
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int s = lane < kScanThreads / 32 ? wsum[lane] : 0;
    s = warp_incl_scan(s);
    if (lane < kScanThreads / 32) wsum[lane] = s;
  }
  __syncthreads();
  int prefix = warp > 0 ? wsum[warp - 1] : 0;
  *total = wsum[kScanThreads / 32 - 1];
  __syncthreads();
  return prefix + inc - v;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ blocksums) {
  const int64_t base = (int64_t)blockIdx.x * PC_SCAN_TILE;
  int s = 0;
#pragma unroll
  for (int r = 0; r < kScanPer; ++r) {
    int64_t i = base + threadIdx.x + (int64_t)r * kScanThreads;
    if (i < n) s += in[i];
  }
  int total;
  (void)block_excl_scan(s, &total);
  if (threadIdx.x == 0) blocksums[blockIdx.x] = total;
}

// One block: exclusive scan of nb block sums in place; out_total receives the sum.
__global__ void k_scan_blocksums(int32_t* __restrict__ bs, int64_t nb, int32_t* __restrict__ out_total) {
  int carry = 0;
  for (int64_t base = 0; base < nb; base += kScanThreads) {
    int64_t i = base + threadIdx.x;
    int v = i < nb ? bs[i] : 0;
    int total;
    int ex = block_excl_scan(v, &total);
    if (i < nb) bs[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) *out_total = carry;
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                             const int32_t* __restrict__ bs) {
  const int64_t base = (int64_t)blockIdx.x * PC_SCAN_TILE + (int64_t)threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
#pragma unroll
  for (int r = 0; r < kScanPer; ++r) {
    v[r] = (base + r < n) ? in[base + r] : 0;
    s += v[r];
  }
  int total;
  int ex = block_excl_scan(s, &total) + bs[blockIdx.x];
#pragma unroll
  for (int r = 0; r < kScanPer; ++r) {
    if (base + r < n) out[base + r] = ex;
    ex += v[r];
  }
}

__global__ void k_bin_scatter(int64_t n, const int32_t* __restrict__ key, const int32_t* __restrict__ slot,
                              const int32_t* __restrict__ start, int32_t* __restrict__ perm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) perm[start[key[i]] + slot[i]] = (int32_t)i;
}

constexpr int kSmallBin = 16;   // a bin of at most this many is sorted by one lane
constexpr int kWarpBin = 256;   // a larger bin up to this many is ranked by the warp (8 per lane)

// Each bin's entries ordered by particle id (ids are distinct). A warp takes 32
// consecutive bins: every lane sorts its own bin when it holds at most kSmallBin
// entries (in registers), then the warp ranks each larger bin together: every
// entry counts the entries of its bin with a smaller id and is written to that
// position. Bins beyond kWarpBin are sorted by insertion by one lane.
__global__ void __launch_bounds__(256) k_bin_order(int64_t nbins, const int32_t* __restrict__ start,
                                                   const int32_t* __restrict__ id, int32_t* __restrict__ perm) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int beg = 0, m = 0;
  if (b < nbins) {
    beg = start[b];
    m = start[b + 1] - beg;
  }
  if (m >= 2 && m <= kSmallBin) {
    int32_t p[kSmallBin], key[kSmallBin];
#pragma unroll
    for (int a = 0; a < kSmallBin; ++a)
      if (a < m) {
        p[a] = perm[beg + a];
        key[a] = id[p[a]];
      }
#pragma unroll
    for (int a = 0; a < kSmallBin; ++a) {
      if (a >= m) break;
      int r = 0;
#pragma unroll
      for (int c = 0; c < kSmallBin; ++c)
        if (c < m && key[c] < key[a]) ++r;
      perm[beg + r] = p[a];
    }
  }
  unsigned big = __ballot_sync(0xffffffffu, m > kSmallBin);
  while (big) {
    const int src = __ffs(big) - 1;
    big &= big - 1;
    const int bb = __shfl_sync(0xffffffffu, beg, src), bm = __shfl_sync(0xffffffffu, m, src);
    if (bm <= kWarpBin) {
      int32_t p[kWarpBin / 32], key[kWarpBin / 32];
#pragma unroll
      for (int u = 0; u < kWarpBin / 32; ++u) {
        const int a = lane + 32 * u;
        p[u] = a < bm ? perm[bb + a] : 0;
        key[u] = a < bm ? id[p[u]] : 0x7fffffff;
      }
      int rank[kWarpBin / 32];
#pragma unroll
      for (int u = 0; u < kWarpBin / 32; ++u) rank[u] = 0;
#pragma unroll
      for (int u2 = 0; u2 < kWarpBin / 32; ++u2) {
        if (32 * u2 >= bm) break;
        for (int sft = 0; sft < 32; ++sft) {
          const int other = __shfl_sync(0xffffffffu, key[u2], sft);
#pragma unroll
          for (int u = 0; u < kWarpBin / 32; ++u) rank[u] += other < key[u] ? 1 : 0;
        }
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kWarpBin / 32; ++u)
        if (lane + 32 * u < bm) perm[bb + rank[u]] = p[u];
      __syncwarp();
    } else if (lane == 0) {
      for (int a = bb + 1; a < bb + bm; ++a) {
        const int32_t q = perm[a];
        const int32_t qid = id[q];
        int c = a - 1;
        while (c >= bb && id[perm[c]] > qid) {
          perm[c + 1] = perm[c];
          --c;
        }
        perm[c + 1] = q;
      }
    }
    __syncwarp();
  }
}

// The same ordering with one warp per bin, for bins that hold tens of entries on
// average (mesh elements): a bin of at most 32 (64) entries is ranked from one (two)
// register tiles, a larger one as in k_bin_order.
__global__ void __launch_bounds__(256) k_bin_order_warp(int64_t nbins, const int32_t* __restrict__ start,
                                                        const int32_t* __restrict__ id, int32_t* __restrict__ perm) {
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= nbins) return;  // warp-uniform
  const int beg = start[b], bm = start[b + 1] - beg;
  if (bm < 2) return;
  if (bm <= 64) {
    const int32_t p0 = lane < bm ? perm[beg + lane] : 0, p1 = lane + 32 < bm ? perm[beg + 32 + lane] : 0;
    const int32_t k0 = lane < bm ? id[p0] : 0x7fffffff, k1 = lane + 32 < bm ? id[p1] : 0x7fffffff;
    int r0 = 0, r1 = 0;
    const int m0 = min(bm, 32);
    for (int sft = 0; sft < m0; ++sft) {
      const int other = __shfl_sync(0xffffffffu, k0, sft);
      r0 += other < k0;
      r1 += other < k1;
    }
    if (bm > 32)
      for (int sft = 0; sft < bm - 32; ++sft) {
        const int other = __shfl_sync(0xffffffffu, k1, sft);
        r0 += other < k0;
        r1 += other < k1;
      }
    __syncwarp();
    if (lane < bm) perm[beg + r0] = p0;
    if (lane + 32 < bm) perm[beg + r1] = p1;
  } else if (bm <= kWarpBin) {
    int32_t p[kWarpBin / 32], key[kWarpBin / 32], rank[kWarpBin / 32];
#pragma unroll
    for (int u = 0; u < kWarpBin / 32; ++u) {
      const int a = lane + 32 * u;
      p[u] = a < bm ? perm[beg + a] : 0;
      key[u] = a < bm ? id[p[u]] : 0x7fffffff;
      rank[u] = 0;
    }
#pragma unroll
    for (int u2 = 0; u2 < kWarpBin / 32; ++u2) {
      if (32 * u2 >= bm) break;
      for (int sft = 0; sft < 32; ++sft) {
        const int other = __shfl_sync(0xffffffffu, key[u2], sft);
#pragma unroll
        for (int u = 0; u < kWarpBin / 32; ++u) rank[u] += other < key[u] ? 1 : 0;
      }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < kWarpBin / 32; ++u)
      if (lane + 32 * u < bm) perm[beg + rank[u]] = p[u];
  } else if (lane == 0) {
    for (int a = beg + 1; a < beg + bm; ++a) {
      const int32_t q = perm[a];
      const int32_t qid = id[q];
      int c = a - 1;
      while (c >= beg && id[perm[c]] > qid) {
        perm[c + 1] = perm[c];
        --c;
      }
      perm[c + 1] = q;
    }
  }
}

}  // namespace

cudaError_t pc_exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* blocksums, cudaStream_t s,
                              int64_t* launches) {
  const int64_t nb = (n + PC_SCAN_TILE - 1) / PC_SCAN_TILE;
  if (nb == 0) return cudaMemsetAsync(out, 0, sizeof(int32_t), s);
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, blocksums);
  k_scan_blocksums<<<1, kScanThreads, 0, s>>>(blocksums, nb, out + n);
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, blocksums);
  *launches += 3;
  return cudaGetLastError();
}

cudaError_t pc_bin_finish(int64_t n, int64_t nbins, const int32_t* key, const int32_t* slot, const int32_t* id,
                          int32_t* cnt, int32_t* start, int32_t* blocksums, int32_t* perm, cudaStream_t s,
                          int64_t* launches) {
  PC_CUDA_TRY(pc_exclusive_scan(cnt, start, nbins, blocksums, s, launches));
  if (n > 0) {
    k_bin_scatter<<<pc_blocks(n, 256), 256, 0, s>>>(n, key, slot, start, perm);
    if (n >= 8 * nbins)
      k_bin_order_warp<<<pc_blocks(32 * nbins, 256), 256, 0, s>>>(nbins, start, id, perm);
    else
      k_bin_order<<<pc_blocks(nbins, 256), 256, 0, s>>>(nbins, start, id, perm);
    *launches += 2;
  }
  return cudaGetLastError();
}
