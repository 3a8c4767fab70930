// Collision step of the particle operator (arXiv 2501.05340, Sec. 2.4, 3.3, 4.3).
//
// Compiled with -fmad=false: every double expression below is evaluated as
// separate IEEE operations in source order, so contact times, velocities and
// positions are bit-identical to a plain FP64 implementation of the same
// formulas. The FP32 pre-filter is conservative by construction (see
// filter_keep) and only decides which pairs reach the exact FP64 test.
//
// Pipeline (one stream, no host synchronisation):
//   keys      cell of every particle, atomic slot in its cell, max |v|^2 and max r
//   bin       exclusive scan of the cell counts, scatter, per-cell order by id
//   gather    sorted FP64 copies of x, v, r, id plus FP32 copies for the filter
//   search    per particle: all candidates j in the neighbour cells, sorted by (t, id)
//   match     round 1 over all particles: commit mutually-earliest pairs
//   finish    one CTA: further rounds over the particles left with candidates
//   respond   impulse, velocity and position update, wrap, write the output state
#include <math.h>

#include "pc_internal.cuh"

namespace {

constexpr int kMaxCap = 32;

__device__ __forceinline__ double minimg(double d) {
  if (d > 0.5) return d - 1.0;
  if (d < -0.5) return d + 1.0;
  return d;
}

__device__ __forceinline__ float minimgf(float d) {
  if (d > 0.5f) return d - 1.0f;
  if (d < -0.5f) return d + 1.0f;
  return d;
}

// y - floor(y) in [0,1]; a tiny negative y rounds it to exactly 1.0, mapped to 0.0.
__device__ __forceinline__ double wrap01(double y) {
  double w = y - floor(y);
  if (w == 1.0) w = 0.0;
  return w;
}

__device__ __forceinline__ int cell_of(double y, int nc) {
  int c = (int)(y * (double)nc);
  c = c < 0 ? 0 : c;
  return c >= nc ? nc - 1 : c;
}

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

__device__ __forceinline__ void raise_status(unsigned long long* counters, int code) {
  atomicMax(&counters[CNT_STATUS], (unsigned long long)code);
}

// Smaller positive root of |dx + t dv| = R with dx = minimg(x_i - x_j), dv = v_i - v_j
// when b < 0, c > 0, b^2 - a c > 0 and the root is <= dt; +inf otherwise.
// Same operations in the same order as the plain definition (Sec. 3.3).
__device__ double contact_time_exact(const double xi[3], const double xj[3], const double vi[3],
                                     const double vj[3], double R, double dt) {
  const double dx0 = minimg(xi[0] - xj[0]);
  const double dx1 = minimg(xi[1] - xj[1]);
  const double dx2 = minimg(xi[2] - xj[2]);
  const double dv0 = vi[0] - vj[0];
  const double dv1 = vi[1] - vj[1];
  const double dv2 = vi[2] - vj[2];
  const double a = (dv0 * dv0 + dv1 * dv1) + dv2 * dv2;
  const double b = (dx0 * dv0 + dx1 * dv1) + dx2 * dv2;
  const double c = ((dx0 * dx0 + dx1 * dx1) + dx2 * dx2) - R * R;
  if (!(b < 0.0)) return CUDART_INF;
  if (!(c > 0.0)) return CUDART_INF;
  const double disc = b * b - a * c;
  if (!(disc > 0.0)) return CUDART_INF;
  const double t = c / (-b + sqrt(disc));
  return t <= dt ? t : CUDART_INF;
}

// Conservative FP32 reject test. A pair accepted by the FP64 test satisfies
// |dx| <= (R + |dv| dt)(1 + O(1e-15)) and dx.dv < 0 (the root formula gives
// c <= 2|b| t and |b| <= |dx||dv|). The FP32 copies of coordinates in [0,1)
// differ from the FP64 values by at most 2^-25, a wrapped difference adds at most
// 2^-25, so |dxf - dx| <= 1.2e-7 per axis (2.1e-7 in norm); each FP32 velocity
// component is within 2^-24 relative, so |dvf - dv| <= 2.1e-7 vmax in norm with
// vmax the largest speed of the step. The test keeps every pair within
// R + |dvf| dt + 4e-7 + 2.5e-7 vmax dt (1e-5 relative slack on top), and every
// pair whose FP32 dx.dv is not clearly positive.
__device__ __forceinline__ bool filter_keep(const float dxf[3], const float dvf[3], float Rf, float dt, float vmax) {
  const float d2 = dxf[0] * dxf[0] + dxf[1] * dxf[1] + dxf[2] * dxf[2];
  const float v2 = dvf[0] * dvf[0] + dvf[1] * dvf[1] + dvf[2] * dvf[2];
  const float vm = sqrtf(v2);
  const float reach = (Rf + vm * dt + 4.0e-7f + 2.5e-7f * vmax * dt) * 1.00001f;
  if (d2 > reach * reach) return false;
  const float bf = dxf[0] * dvf[0] + dxf[1] * dvf[1] + dxf[2] * dvf[2];
  const float bslack = (4.0e-7f + 1.0e-6f * sqrtf(d2)) * (vm + vmax);
  return !(bf > bslack);
}

// ------------------------------------------------------------------ keys

__global__ void k_collide_keys(int64_t n, const double* __restrict__ x, const double* __restrict__ v,
                               const double* __restrict__ r, const double* __restrict__ m, int nc,
                               int32_t* __restrict__ key, int32_t* __restrict__ slot, int32_t* __restrict__ cnt,
                               unsigned long long* __restrict__ counters) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v2 = 0.0, rr = 0.0;
  if (i < n) {
    const double x0 = x[i], x1 = x[n + i], x2 = x[2 * n + i];
    const double v0 = v[i], v1 = v[n + i], vv2 = v[2 * n + i];
    rr = r[i];
    const double mm = m[i];
    const bool ok = (x0 >= 0.0 && x0 < 1.0) && (x1 >= 0.0 && x1 < 1.0) && (x2 >= 0.0 && x2 < 1.0) &&
                    (rr > 0.0 && rr < 0.25) && (mm > 0.0 && mm < CUDART_INF) && isfinite(v0) && isfinite(v1) &&
                    isfinite(vv2);
    if (!ok) raise_status(counters, PC_EINVAL);
    const int k = (cell_of(x2, nc) * nc + cell_of(x1, nc)) * nc + cell_of(x0, nc);
    key[i] = k;
    slot[i] = atomicAdd(&cnt[k], 1);
    v2 = (v0 * v0 + v1 * v1) + vv2 * vv2;
    if (!(v2 < CUDART_INF)) v2 = 0.0;
    if (!(rr > 0.0 && rr < 0.25)) rr = 0.0;
  }
  pc_block_max2(&counters[CNT_VMAX2], v2, &counters[CNT_RMAX], rr);
}

// ------------------------------------------------------------------ gather

__global__ void k_collide_gather(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ x,
                                 const double* __restrict__ v, const double* __restrict__ r,
                                 const int32_t* __restrict__ id, double* __restrict__ sx, double* __restrict__ sv,
                                 double* __restrict__ sr, int32_t* __restrict__ sid, float* __restrict__ sxf,
                                 float* __restrict__ svf, float* __restrict__ srf) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t p = perm[k];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double xa = x[a * n + p], va = v[a * n + p];
    sx[a * n + k] = xa;
    sv[a * n + k] = va;
    sxf[a * n + k] = (float)xa;
    svf[a * n + k] = (float)va;
  }
  const double rr = r[p];
  sr[k] = rr;
  srf[k] = (float)rr;
  sid[k] = id[p];
}

// ------------------------------------------------------------------ search

struct SearchArgs {
  int64_t n;
  int nc;
  int cap;
  double dt;
  const double *sx, *sv, *sr;
  const int32_t* sid;
  const float *sxf, *svf, *srf;
  const int32_t* start;
  int32_t* cand_j;
  double* cand_t;
  int32_t* ncand;
  int32_t* best;
  unsigned long long* counters;
};

// Neighbour cells searched on each side: the largest possible reach
// 2 r_max + 2 v_max dt (Sec. 4.3, halo criterion) in units of the cell side,
// plus one for the rounding of cell indices.
__device__ __forceinline__ int stencil_radius(const unsigned long long* counters, int nc, double dt, double* reach) {
  const double v2 = __longlong_as_double((long long)counters[CNT_VMAX2]);
  const double rm = __longlong_as_double((long long)counters[CNT_RMAX]);
  const double re = (2.0 * rm + 2.0 * sqrt(v2) * dt) * (1.0 + 1e-9) + 1e-12;
  *reach = re;
  double s = floor(re * (double)nc * (1.0 + 1e-9)) + 1.0;
  if (s > (double)nc) s = (double)nc;
  return (int)s;
}

constexpr int kPassCap = 64;  // distance-test passes queued per warp
constexpr int kSurvCap = 64;  // filter survivors queued per warp
constexpr unsigned kFull = 0xffffffffu;

// Exact FP64 contact time of the pair (k, j) of the sorted arrays.
__device__ __forceinline__ double solve_pair(const SearchArgs& A, int64_t k, int64_t j) {
  const int64_t n = A.n;
  const double xi[3] = {A.sx[k], A.sx[n + k], A.sx[2 * n + k]};
  const double vi[3] = {A.sv[k], A.sv[n + k], A.sv[2 * n + k]};
  const double xj[3] = {A.sx[j], A.sx[n + j], A.sx[2 * n + j]};
  const double vj[3] = {A.sv[j], A.sv[n + j], A.sv[2 * n + j]};
  return contact_time_exact(xi, xj, vi, vj, A.sr[k] + A.sr[j], A.dt);
}

// Insertion into a list sorted by (t, id), keeping the cap first.
__device__ __forceinline__ void insert_sorted(double* lt, int* lj, int& cnt, int cap, double t, int j,
                                              const int32_t* sid) {
  const int jid = sid[j];
  int pos = cnt;
  while (pos > 0 && (lt[pos - 1] > t || (lt[pos - 1] == t && sid[lj[pos - 1]] > jid))) --pos;
  if (pos >= cap) return;
  const int last = cnt < cap ? cnt : cap - 1;
  for (int q = last; q > pos; --q) {
    lt[q] = lt[q - 1];
    lj[q] = lj[q - 1];
  }
  lt[pos] = t;
  lj[pos] = j;
  if (cnt < cap) ++cnt;
}

// Morton (Z-order) code of a cell with coordinates below 1024: bit b of cx, cy, cz to
// bit 3b, 3b+1, 3b+2.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Rank key of sorted particle j along the curve of the first-found pair selection:
// (Morton code of its cell, id).
__device__ __forceinline__ unsigned long long sfc_key(const double* __restrict__ sx, const int32_t* __restrict__ sid,
                                                      int64_t n, int nc, int64_t j) {
  const uint32_t code = spread3((uint32_t)cell_of(sx[j], nc)) | (spread3((uint32_t)cell_of(sx[n + j], nc)) << 1) |
                        (spread3((uint32_t)cell_of(sx[2 * n + j], nc)) << 2);
  return ((unsigned long long)code << 32) | (uint32_t)sid[j];
}

// Insertion into a list sorted by the partner's rank key (first-found selection).
__device__ __forceinline__ void insert_by_key(double* lt, int* lj, unsigned long long* lk, int& cnt, int cap,
                                              double t, int j, unsigned long long key) {
  int pos = cnt;
  while (pos > 0 && lk[pos - 1] > key) --pos;
  if (pos >= cap) return;
  const int last = cnt < cap ? cnt : cap - 1;
  for (int q = last; q > pos; --q) {
    lt[q] = lt[q - 1];
    lj[q] = lj[q - 1];
    lk[q] = lk[q - 1];
  }
  lt[pos] = t;
  lj[pos] = j;
  lk[pos] = key;
  if (cnt < cap) ++cnt;
}

// Per-warp queues of the contact search in shared memory.
struct SearchQueue {
  float dx[kPassCap], dy[kPassCap], dz[kPassCap];  // offsets of the queued distance-test passes
  int j[kPassCap], own[kPassCap];                  // candidate and owning lane
  int sown[kSurvCap], sj[kSurvCap];                // filter survivors
  double st[kSurvCap];                             // their FP64 roots
};

// Thread per particle (sorted by cell), the warp's lanes in lockstep. The stencil is
// taken row by row; a row's 2 s + 1 cells along x are one contiguous range of the
// sorted arrays, or two where the row wraps. Each candidate first takes a distance
// test against a reach that no pair of this particle exceeds in filter_keep (the
// particle's radius plus the largest one, its speed plus the largest one, with
// margins above the FP32 rounding); the passes are queued per warp and, 32 at a
// time, go through the certified filter with one pass per lane. Its survivors are
// queued again and solved exactly in FP64 by the warp's lanes together (on this GPU
// an FP64 instruction takes a warp 64 pipe cycles whatever the number of active
// lanes); every lane then inserts its own roots into its list sorted by (t, id),
// which does not depend on the order in which they were found. kSfc: the lists are
// sorted by the partner's rank key instead (the paper's first-found selection; the
// matching then takes, for every particle, its first free candidate in that order).
template <bool kSfc>
__global__ void __launch_bounds__(256, 3) k_search(SearchArgs A) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  const int nc = A.nc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  // stencil radius and speed and radius bounds from the step's maxima, once per block
  __shared__ int s_sh;
  __shared__ float vmaxf_sh, rmaxf_sh;
  __shared__ SearchQueue queues[8];
  SearchQueue& Q = queues[warp];
  __shared__ int stat_sh[3];  // candidates found, FP64 solves, largest list
  if (threadIdx.x == 0) {
    stat_sh[0] = stat_sh[1] = stat_sh[2] = 0;
    double reach;
    s_sh = stencil_radius(A.counters, A.nc, A.dt, &reach);
    vmaxf_sh = (float)sqrt(__longlong_as_double((long long)A.counters[CNT_VMAX2])) * 1.000001f;
    rmaxf_sh = (float)__longlong_as_double((long long)A.counters[CNT_RMAX]) * 1.000001f;
    if (blockIdx.x == 0) {
      atomicMax(&A.counters[CNT_STENCIL], (unsigned long long)s_sh);
      if (!(reach < 0.5)) raise_status(A.counters, PC_EINVAL);
    }
  }
  __syncthreads();
  const int s = s_sh;
  const float dtf = (float)A.dt * 1.000001f;
  const float vmaxf = vmaxf_sh;
  const bool live = k < n;
  const int64_t kw = (int64_t)blockIdx.x * blockDim.x + 32 * warp;  // the warp's first particle
  int found = 0, solves = 0, cnt = 0;
  double lt[kMaxCap];
  int lj[kMaxCap];
  unsigned long long lk[kSfc ? kMaxCap : 1];
  float xf[3] = {0.0f, 0.0f, 0.0f}, vf[3] = {0.0f, 0.0f, 0.0f}, rf = 0.0f, rl2 = -1.0f;
  int cx = 0, cy = 0, cz = 0;
  if (live) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      xf[a] = A.sxf[a * n + k];
      vf[a] = A.svf[a * n + k];
    }
    rf = A.srf[k];
    cx = cell_of(A.sx[k], nc);
    cy = cell_of(A.sx[n + k], nc);
    cz = cell_of(A.sx[2 * n + k], nc);
    const float vkf = sqrtf(vf[0] * vf[0] + vf[1] * vf[1] + vf[2] * vf[2]) * 1.000001f;
    const float rhi = ((rf + rmaxf_sh) + (vkf + vmaxf) * dtf) * 1.00002f + 4.0e-7f + 2.5e-7f * vmaxf * dtf;
    rl2 = rhi * rhi * 1.0001f;
  }
  int np = 0, ns = 0;  // queued passes and survivors (the same in every lane)

  // the queued survivors' FP64 roots, by the lanes together; each lane then inserts its own
  auto flush_survivors = [&]() {
    for (int e = lane; e < ns; e += 32) {
      Q.st[e] = solve_pair(A, kw + Q.sown[e], Q.sj[e]);
      ++solves;
    }
    __syncwarp();
    for (int e = 0; e < ns; ++e) {
      if (Q.sown[e] != lane) continue;
      const double t = Q.st[e];
      if (t <= A.dt) {
        ++found;
        if constexpr (kSfc)
          insert_by_key(lt, lj, lk, cnt, A.cap, t, Q.sj[e], sfc_key(A.sx, A.sid, n, nc, Q.sj[e]));
        else
          insert_sorted(lt, lj, cnt, A.cap, t, Q.sj[e], A.sid);
      }
    }
    __syncwarp();
    ns = 0;
  };
  // the certified filter on the first m <= 32 queued passes, one per lane
  auto filter_passes = [&](int m) {
    const int own = lane < m ? Q.own[lane] : lane;
    const float vo0 = __shfl_sync(kFull, vf[0], own), vo1 = __shfl_sync(kFull, vf[1], own),
                vo2 = __shfl_sync(kFull, vf[2], own), ro = __shfl_sync(kFull, rf, own);
    bool keep = false;
    int j = 0;
    if (lane < m) {
      j = Q.j[lane];
      const float dxf[3] = {Q.dx[lane], Q.dy[lane], Q.dz[lane]};
      const float dvf[3] = {vo0 - A.svf[j], vo1 - A.svf[n + j], vo2 - A.svf[2 * n + j]};
      keep = filter_keep(dxf, dvf, ro + A.srf[j], dtf, vmaxf);
    }
    const unsigned bal = __ballot_sync(kFull, keep);
    if (keep) {
      const int p = ns + __popc(bal & below);
      Q.sown[p] = own;
      Q.sj[p] = j;
    }
    ns += __popc(bal);
    __syncwarp();
    if (ns > kSurvCap - 32) flush_survivors();
  };

  const int span = 2 * s + 1;
  const bool full = span >= nc;  // the stencil covers the whole axis: visit every cell once
  const int cnt_ax = full ? nc : span;
  // per-axis bases of the candidate arrays and a 32-bit own index for the inner loop
  const float* __restrict__ sx0 = A.sxf;
  const float* __restrict__ sx1 = A.sxf + n;
  const float* __restrict__ sx2 = A.sxf + 2 * n;
  const int k32 = live ? (int)k : -1;
  for (int oz = 0; oz < cnt_ax; ++oz) {
    for (int oy = 0; oy < cnt_ax; ++oy) {
      int b1 = 0, e1 = 0, b2 = 0, e2 = 0;
      if (live) {
        const int zc = full ? oz : wrapi(cz - s + oz, nc);
        const int yc = full ? oy : wrapi(cy - s + oy, nc);
        const int64_t row = ((int64_t)zc * nc + yc) * nc;
        const int xl = cx - s, xh = cx + s;
        if (full) {
          b1 = A.start[row];
          e1 = A.start[row + nc];
        } else if (xl >= 0 && xh < nc) {
          b1 = A.start[row + xl];
          e1 = A.start[row + xh + 1];
        } else if (xl < 0) {
          b1 = A.start[row + xl + nc];
          e1 = A.start[row + nc];
          b2 = A.start[row];
          e2 = A.start[row + xh + 1];
        } else {
          b1 = A.start[row + xl];
          e1 = A.start[row + nc];
          b2 = A.start[row];
          e2 = A.start[row + xh - nc + 1];
        }
      }
      const int l1 = e1 - b1, len = l1 + (e2 - b2);
      const int m = __reduce_max_sync(kFull, len);
      for (int t = 0; t < m; ++t) {
        const int j = t < l1 ? b1 + t : b2 + (t - l1);
        bool pass = false;
        float dx = 0.0f, dy = 0.0f, dz = 0.0f;
        if (t < len && j != k32) {
          dx = minimgf(xf[0] - sx0[j]);
          dy = minimgf(xf[1] - sx1[j]);
          dz = minimgf(xf[2] - sx2[j]);
          pass = !(dx * dx + dy * dy + dz * dz > rl2);
        }
        const unsigned bal = __ballot_sync(kFull, pass);
        if (pass) {
          const int p = np + __popc(bal & below);
          Q.dx[p] = dx;
          Q.dy[p] = dy;
          Q.dz[p] = dz;
          Q.j[p] = j;
          Q.own[p] = lane;
        }
        np += __popc(bal);
        if (np >= 32) {
          __syncwarp();
          filter_passes(32);
          // move the passes beyond the first 32 to the front
          const bool mv = lane < np - 32;
          float mx = 0.0f, my = 0.0f, mz = 0.0f;
          int mj = 0, mo = 0;
          if (mv) {
            mx = Q.dx[32 + lane];
            my = Q.dy[32 + lane];
            mz = Q.dz[32 + lane];
            mj = Q.j[32 + lane];
            mo = Q.own[32 + lane];
          }
          __syncwarp();
          if (mv) {
            Q.dx[lane] = mx;
            Q.dy[lane] = my;
            Q.dz[lane] = mz;
            Q.j[lane] = mj;
            Q.own[lane] = mo;
          }
          __syncwarp();
          np -= 32;
        }
      }
    }
  }
  __syncwarp();
  if (np > 0) filter_passes(np);
  if (ns > 0) flush_survivors();
  if (live) {
    for (int q = 0; q < cnt; ++q) {
      A.cand_j[(int64_t)q * n + k] = lj[q];
      A.cand_t[(int64_t)q * n + k] = lt[q];
    }
    A.ncand[k] = cnt;
    A.best[k] = cnt > 0 ? lj[0] : -1;
    if (found > A.cap) raise_status(A.counters, PC_ECAPACITY);
  }
  // statistics: warp sums into shared counters, one global atomic per block
  int fsum = found, ssum = solves, fmx = found;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fsum += __shfl_xor_sync(0xffffffffu, fsum, o);
    ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
    fmx = max(fmx, __shfl_xor_sync(0xffffffffu, fmx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (fsum) atomicAdd(&stat_sh[0], fsum);
    if (ssum) atomicAdd(&stat_sh[1], ssum);
    if (fmx) atomicMax(&stat_sh[2], fmx);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (stat_sh[0]) atomicAdd(&A.counters[CNT_CANDS], (unsigned long long)stat_sh[0]);
    if (stat_sh[1]) atomicAdd(&A.counters[CNT_SOLVES], (unsigned long long)stat_sh[1]);
    if (stat_sh[2] && (unsigned long long)stat_sh[2] > *(volatile unsigned long long*)&A.counters[CNT_MAXCAND])
      atomicMax(&A.counters[CNT_MAXCAND], (unsigned long long)stat_sh[2]);
  }
}

// ------------------------------------------------------------------ matching

struct MatchArgs {
  int64_t n;
  int cap;
  const int32_t* cand_j;
  const double* cand_t;
  const int32_t* ncand;
  int32_t* best;
  const int32_t* sid;
  int32_t* partner;
  double* tcoll;
  int32_t* work;
  int32_t *pair_lo, *pair_hi;
  double* pair_t;
  unsigned long long* counters;
};

__device__ __forceinline__ void record_pair(const MatchArgs& M, int64_t k, int64_t b, double t) {
  const int32_t ik = M.sid[k], ib = M.sid[b];
  if (ik < ib) {
    const unsigned long long q = atomicAdd(&M.counters[CNT_PAIRS], 1ull);
    M.pair_lo[q] = ik;
    M.pair_hi[q] = ib;
    M.pair_t[q] = t;
  }
}

// Round 1: every particle's earliest candidate is its pick; mutual picks collide.
// The pair list and the work list take their slots once per warp (the pair list is
// read back sorted, the work list's order does not matter).
__global__ void k_match_first(MatchArgs M) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const bool in = k < M.n;
  int b = -1;
  bool mutual = false;
  if (in) {
    b = M.best[k];
    mutual = b >= 0 && M.best[b] == (int)k;
  }
  double t = CUDART_INF;
  bool rec = false;
  if (mutual) {
    t = M.cand_t[k];
    rec = M.sid[k] < M.sid[b];
  }
  if (in) {
    M.partner[k] = mutual ? b : -1;
    M.tcoll[k] = t;
  }
  const unsigned br = __ballot_sync(0xffffffffu, rec);
  if (br) {
    const int lead = __ffs(br) - 1;
    unsigned long long base = 0;
    if (lane == lead) {
      base = atomicAdd(&M.counters[CNT_PAIRS], (unsigned long long)__popc(br));
      if (*(volatile unsigned long long*)&M.counters[CNT_ROUNDS] == 0ull) atomicMax(&M.counters[CNT_ROUNDS], 1ull);
    }
    base = __shfl_sync(0xffffffffu, base, lead);
    if (rec) {
      const unsigned long long q = base + __popc(br & below);
      M.pair_lo[q] = M.sid[k];
      M.pair_hi[q] = M.sid[b];
      M.pair_t[q] = t;
    }
  }
  const bool wk = in && !mutual && b >= 0;
  const unsigned bw = __ballot_sync(0xffffffffu, wk);
  if (bw) {
    const int lead = __ffs(bw) - 1;
    unsigned long long base = 0;
    if (lane == lead) base = atomicAdd(&M.counters[CNT_WORK], (unsigned long long)__popc(bw));
    base = __shfl_sync(0xffffffffu, base, lead);
    if (wk) M.work[base + __popc(bw & below)] = (int32_t)k;
  }
}

// Further rounds in one CTA over the particles that still had candidates after
// round 1: pick the earliest candidate that is still free, commit mutual picks.
// Each round that has a pick commits at least the globally earliest remaining
// pair, so the loop ends after at most |work| + 1 rounds; the cap is a guard.
constexpr int kFinishThreads = 1024;

__global__ void __launch_bounds__(kFinishThreads) k_match_finish(MatchArgs M) {
  const int64_t nw = (int64_t)M.counters[CNT_WORK];
  if (nw == 0) return;
  const int64_t n = M.n;
  unsigned long long rounds = M.counters[CNT_ROUNDS];
  for (int64_t r = 0;; ++r) {
    int any = 0;
    for (int64_t w = threadIdx.x; w < nw; w += kFinishThreads) {
      const int64_t k = M.work[w];
      if (M.partner[k] >= 0) continue;
      const int c = M.ncand[k];
      int nb = -1;
      for (int q = 0; q < c; ++q) {
        const int j = M.cand_j[(int64_t)q * n + k];
        if (M.partner[j] < 0) {
          nb = j;
          break;
        }
      }
      M.best[k] = nb;
      any |= nb >= 0;
    }
    if (!__syncthreads_or(any)) break;
    if (r > nw + 1) {
      if (threadIdx.x == 0) raise_status(M.counters, PC_ENOCONVERGE);
      break;
    }
    int committed = 0;
    for (int64_t w = threadIdx.x; w < nw; w += kFinishThreads) {
      const int64_t k = M.work[w];
      if (M.partner[k] >= 0) continue;
      const int b = M.best[k];
      if (b >= 0 && M.best[b] == (int)k) {
        const int c = M.ncand[k];
        double t = CUDART_INF;
        for (int q = 0; q < c; ++q)
          if (M.cand_j[(int64_t)q * n + k] == b) {
            t = M.cand_t[(int64_t)q * n + k];
            break;
          }
        M.partner[k] = b;
        M.tcoll[k] = t;
        record_pair(M, k, b, t);
        committed = 1;
      }
    }
    if (__syncthreads_or(committed)) ++rounds;
  }
  if (threadIdx.x == 0) M.counters[CNT_ROUNDS] = rounds;
}

// ------------------------------------------------------------------ respond

struct RespondArgs {
  int64_t n;
  double dt, e;
  const double *sx, *sv, *sr;
  const int32_t* sid;
  const int32_t* partner;
  const double* tcoll;
  const int32_t* perm;
  const double* m_in;
  const double* q_in;
  double *x_out, *v_out, *r_out, *m_out, *q_out;
  int32_t* id_out;
  // friction and rotation (k_respond_rot): angular velocities in input order / sorted order
  double mu;
  const double* w_in;
  double* w_out;
  int32_t* list;                  // [n]: sorted indices of the colliding particles (k_respond)
  unsigned long long* counters;   // CNT_RESP counts them
};

// Frictionless hard-sphere response (Sec. 2.4) from the particle's own side:
// s = dx + t dv (from partner to self), n = -s/|s|, v_r.n, m_r = m_i m_j/(m_i + m_j),
// J = -m_r (1 + e) v_r.n, v' = v + (J/m_i) n, x' = x + t v + (dt - t) v' (Sec. 3.3).
__device__ __forceinline__ void pair_response(const RespondArgs& R, int64_t k, int32_t j, double mi, double xo[3],
                                              double vo[3]) {
  const int64_t n = R.n;
  const double xi[3] = {R.sx[k], R.sx[n + k], R.sx[2 * n + k]};
  const double vi[3] = {R.sv[k], R.sv[n + k], R.sv[2 * n + k]};
  const double t = R.tcoll[k];
  const double mj = R.m_in[R.perm[j]];
  double dx[3], dv[3], s[3], nr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    dx[a] = minimg(xi[a] - R.sx[a * n + j]);
    dv[a] = vi[a] - R.sv[a * n + j];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) s[a] = dx[a] + t * dv[a];
  const double sl = sqrt((s[0] * s[0] + s[1] * s[1]) + s[2] * s[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) nr[a] = -s[a] / sl;
  const double vrn = (dv[0] * nr[0] + dv[1] * nr[1]) + dv[2] * nr[2];
  const double mr = (mi * mj) / (mi + mj);
  const double J = -mr * (1.0 + R.e) * vrn;
  const double gi = J / mi;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double vnew = vi[a] + gi * nr[a];
    vo[a] = vnew;
    xo[a] = (xi[a] + t * vi[a]) + (R.dt - t) * vnew;
  }
}

// Free particles fly; colliding particles go to a list (slots once per warp) and
// k_respond_pairs computes their responses with every lane of a warp busy (an FP64
// instruction takes a warp 64 pipe cycles on this GPU whatever the number of
// active lanes). The response of each particle is computed from its own side.
__global__ void __launch_bounds__(256) k_respond(RespondArgs R) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = R.n;
  const int lane = threadIdx.x & 31;
  bool col = false;
  if (k < n) {
    const int64_t p = R.perm[k];
    const int32_t j = R.partner[k];
    const double mi = R.m_in[p];
    if (j < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double vi = R.sv[a * n + k];
        R.x_out[a * n + k] = wrap01(R.sx[a * n + k] + R.dt * vi);
        R.v_out[a * n + k] = vi;
      }
    } else {
      col = true;
    }
    R.r_out[k] = R.sr[k];
    R.m_out[k] = mi;
    R.id_out[k] = R.sid[k];
    if (R.q_out) {
#pragma unroll
      for (int c = 0; c < 4; ++c) R.q_out[c * n + k] = R.q_in[c * n + p];
    }
  }
  const unsigned bc = __ballot_sync(0xffffffffu, col);
  if (bc) {
    const int lead = __ffs(bc) - 1;
    unsigned long long base = 0;
    if (lane == lead) base = atomicAdd(&R.counters[CNT_RESP], (unsigned long long)__popc(bc));
    base = __shfl_sync(0xffffffffu, base, lead);
    if (col) R.list[base + __popc(bc & ((1u << lane) - 1u))] = (int32_t)k;
  }
}

// Responses of the listed colliding particles, grid-stride over the list.
__global__ void __launch_bounds__(256) k_respond_pairs(RespondArgs R) {
  const int64_t cnt = (int64_t)R.counters[CNT_RESP];
  const int64_t n = R.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kk = R.list[i];
    double xo[3], vo[3];
    pair_response(R, kk, R.partner[kk], R.m_in[R.perm[kk]], xo, vo);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R.x_out[a * n + kk] = wrap01(xo[a]);
      R.v_out[a * n + kk] = vo[a];
    }
  }
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// The response with friction and rotation of sorted particle k with partner j (see
// k_respond_rot).
__device__ __forceinline__ void pair_response_rot(const RespondArgs& R, int64_t k, int32_t j, double xo[3],
                                                  double vo[3], double wo[3]) {
  const int64_t n = R.n;
  const int64_t p = R.perm[k];
  const double mi = R.m_in[p];
  const double xi[3] = {R.sx[k], R.sx[n + k], R.sx[2 * n + k]};
  const double vi[3] = {R.sv[k], R.sv[n + k], R.sv[2 * n + k]};
  const double wi[3] = {R.w_in[p], R.w_in[n + p], R.w_in[2 * n + p]};
  const double t = R.tcoll[k];
  const int64_t pj = R.perm[j];
  const double mj = R.m_in[pj];
  double dx[3], dv[3], s[3], nr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    dx[a] = minimg(xi[a] - R.sx[a * n + j]);
    dv[a] = vi[a] - R.sv[a * n + j];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) s[a] = dx[a] + t * dv[a];
  const double sl = sqrt((s[0] * s[0] + s[1] * s[1]) + s[2] * s[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) nr[a] = -s[a] / sl;
  const double vrn = (dv[0] * nr[0] + dv[1] * nr[1]) + dv[2] * nr[2];
  const double mr = (mi * mj) / (mi + mj);
  const double Jn = -mr * (1.0 + R.e) * vrn;
  const double wj[3] = {R.w_in[pj], R.w_in[n + pj], R.w_in[2 * n + pj]};
  const double ri = R.sr[k], rj = R.sr[j];
  const bool self_lo = R.sid[k] < R.sid[j];
  double cl[3], ch[3], vc[3];
  cross3(self_lo ? wi : wj, nr, cl);
  cross3(self_lo ? wj : wi, nr, ch);
  const double rl = self_lo ? ri : rj, rh = self_lo ? rj : ri;
#pragma unroll
  for (int a = 0; a < 3; ++a) vc[a] = (dv[a] + rl * cl[a]) + rh * ch[a];
  const double vcn = (vc[0] * nr[0] + vc[1] * nr[1]) + vc[2] * nr[2];
  double vt[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) vt[a] = vc[a] - vcn * nr[a];
  const double vtl = sqrt((vt[0] * vt[0] + vt[1] * vt[1]) + vt[2] * vt[2]);
  double Jt = 0.0, tv[3] = {0.0, 0.0, 0.0};
  if (vtl > 0.0) {
    const double slide = R.mu * Jn, stick = -(2.0 / 7.0) * (1.0 + R.e) * mr * vtl;
    Jt = slide > stick ? slide : stick;
#pragma unroll
    for (int a = 0; a < 3; ++a) tv[a] = vt[a] / vtl;
  }
  const double gn = Jn / mi, gt = Jt / mi;
  double nt[3];
  cross3(nr, tv, nt);
  const double inertia = 0.4 * mi * ri * ri;
  const double gw = (ri * Jt) / inertia;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double vnew = (vi[a] + gn * nr[a]) + gt * tv[a];
    vo[a] = vnew;
    wo[a] = wi[a] + gw * nt[a];
    xo[a] = (xi[a] + t * vi[a]) + (R.dt - t) * vnew;
  }
}

// Response with Coulomb friction and rotation (Sec. 2.4) from the particle's own side
// (it is particle 1, n from it to its partner): J = J_n n + J_t t, J_n = -m_r (1+e) v_r.n,
// contact-point velocity v_c = v_r + r_1 w_1 x n + r_2 w_2 x n with the two rotational
// terms added in id order (lower first, so both sides see the same bits up to sign),
// v_rt = v_c - (v_c.n) n, J_t = max(mu J_n, -(2/7)(1+e) m_r |v_rt|), t = v_rt/|v_rt| (no
// tangential impulse when |v_rt| = 0); v' = v + (J_n/m) n + (J_t/m) t and
// w' = w + (r J_t / I)(n x t) with I = (2/5) m r^2; x' = x + t v + (dt - t) v'. The
// colliding particles of a block are computed densely, as in k_respond.
__global__ void __launch_bounds__(256) k_respond_rot(RespondArgs R) {
  __shared__ int q_cnt;
  __shared__ int q_k[256];
  if (threadIdx.x == 0) q_cnt = 0;
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = R.n;
  if (k < n) {
    const int64_t p = R.perm[k];
    const int32_t j = R.partner[k];
    if (j < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double vi = R.sv[a * n + k];
        R.x_out[a * n + k] = wrap01(R.sx[a * n + k] + R.dt * vi);
        R.v_out[a * n + k] = vi;
        R.w_out[a * n + k] = R.w_in[a * n + p];
      }
    } else {
      q_k[atomicAdd(&q_cnt, 1)] = threadIdx.x;
    }
    R.r_out[k] = R.sr[k];
    R.m_out[k] = R.m_in[p];
    R.id_out[k] = R.sid[k];
    if (R.q_out) {
#pragma unroll
      for (int c = 0; c < 4; ++c) R.q_out[c * n + k] = R.q_in[c * n + p];
    }
  }
  __syncthreads();
  const int nq = q_cnt;
  for (int e = threadIdx.x; e < nq; e += blockDim.x) {
    const int64_t kk = (int64_t)blockIdx.x * blockDim.x + q_k[e];
    double xo[3], vo[3], wo[3];
    pair_response_rot(R, kk, R.partner[kk], xo, vo, wo);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R.x_out[a * n + kk] = wrap01(xo[a]);
      R.v_out[a * n + kk] = vo[a];
      R.w_out[a * n + kk] = wo[a];
    }
  }
}

}  // namespace

cudaError_t pc_match_launch(pc_ctx* ctx, int64_t n) {
  MatchArgs M;
  M.n = n;
  M.cap = ctx->cap;
  M.cand_j = ctx->cand_j;
  M.cand_t = ctx->cand_t;
  M.ncand = ctx->ncand;
  M.best = ctx->best;
  M.sid = ctx->sid;
  M.partner = ctx->partner;
  M.tcoll = ctx->tcoll;
  M.work = ctx->work;
  M.pair_lo = ctx->pair_lo;
  M.pair_hi = ctx->pair_hi;
  M.pair_t = ctx->pair_t;
  M.counters = ctx->counters;
  const int tm = pc_phase_begin(ctx, PC_PH_MATCH);
  k_match_first<<<pc_blocks(n, 256), 256, 0, ctx->stream>>>(M);
  k_match_finish<<<1, kFinishThreads, 0, ctx->stream>>>(M);
  ctx->launches += 2;
  pc_phase_end(ctx, tm);
  return cudaGetLastError();
}

pc_status pc_collide_impl(pc_ctx* ctx, const pc_particles* in, pc_particles* out, double dt, const double* w_in,
                          double* w_out, double mu) {
  const int64_t n = in->n;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaSuccess;
  e = cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned long long) * CNT_N, st);
  if (e == cudaSuccess && n == 0) return PC_OK;
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->cnt, 0, sizeof(int32_t) * (size_t)ctx->ncell, st);
  if (e != cudaSuccess) goto fail;
  {
    const int tb = pc_phase_begin(ctx, PC_PH_BIN);
    k_collide_keys<<<pc_blocks(n, 256), 256, 0, st>>>(n, in->x, in->v, in->r, in->m, ctx->nc, ctx->key, ctx->slot,
                                                       ctx->cnt, ctx->counters);
    ctx->launches += 1;
    e = pc_bin_finish(n, ctx->ncell, ctx->key, ctx->slot, in->id, ctx->cnt, ctx->start, ctx->blocksums, ctx->perm, st,
                      &ctx->launches);
    pc_phase_end(ctx, tb);
  }
  if (e != cudaSuccess) goto fail;
  {
    const int tg = pc_phase_begin(ctx, PC_PH_GATHER);
    k_collide_gather<<<pc_blocks(n, 256), 256, 0, st>>>(n, ctx->perm, in->x, in->v, in->r, in->id, ctx->sx, ctx->sv,
                                                         ctx->sr, ctx->sid, ctx->sxf, ctx->svf, ctx->srf);
    ctx->launches += 1;
    pc_phase_end(ctx, tg);
  }
  {
    SearchArgs A;
    A.n = n;
    A.nc = ctx->nc;
    A.cap = ctx->cap;
    A.dt = dt;
    A.sx = ctx->sx;
    A.sv = ctx->sv;
    A.sr = ctx->sr;
    A.sid = ctx->sid;
    A.sxf = ctx->sxf;
    A.svf = ctx->svf;
    A.srf = ctx->srf;
    A.start = ctx->start;
    A.cand_j = ctx->cand_j;
    A.cand_t = ctx->cand_t;
    A.ncand = ctx->ncand;
    A.best = ctx->best;
    A.counters = ctx->counters;
    const int ts = pc_phase_begin(ctx, PC_PH_SEARCH);
    if (ctx->pair_policy == PC_PAIRS_SFC_FIRST)
      k_search<true><<<pc_blocks(n, 256), 256, 0, st>>>(A);
    else
      k_search<false><<<pc_blocks(n, 256), 256, 0, st>>>(A);
    ctx->launches += 1;
    pc_phase_end(ctx, ts);
  }
  e = pc_match_launch(ctx, n);
  if (e != cudaSuccess) goto fail;
  {
    RespondArgs R;
    R.n = n;
    R.dt = dt;
    R.e = ctx->cfg.restitution;
    R.sx = ctx->sx;
    R.sv = ctx->sv;
    R.sr = ctx->sr;
    R.sid = ctx->sid;
    R.partner = ctx->partner;
    R.tcoll = ctx->tcoll;
    R.perm = ctx->perm;
    R.m_in = in->m;
    R.q_in = in->q;
    R.x_out = out->x;
    R.v_out = out->v;
    R.r_out = out->r;
    R.m_out = out->m;
    R.q_out = in->q ? out->q : nullptr;
    R.id_out = out->id;
    R.mu = mu;
    R.w_in = w_in;
    R.w_out = w_out;
    R.list = ctx->work;  // the matching's work list is spent by now
    R.counters = ctx->counters;
    const int tr = pc_phase_begin(ctx, PC_PH_RESPOND);
    if (w_in) {
      k_respond_rot<<<pc_blocks(n, 256), 256, 0, st>>>(R);
      ctx->launches += 1;
    } else {
      k_respond<<<pc_blocks(n, 256), 256, 0, st>>>(R);
      const int gp = pc_blocks(n, 256) < 4096 ? pc_blocks(n, 256) : 4096;
      k_respond_pairs<<<gp, 256, 0, st>>>(R);
      ctx->launches += 2;
    }
    pc_phase_end(ctx, tr);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
fail:
  snprintf(ctx->err, sizeof(ctx->err), "pc_collide: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}
