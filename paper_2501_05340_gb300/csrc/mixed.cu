// Mixed-precision path of the particle operator (arXiv 2501.05340 operator with
// FP32 cell-relative storage): quantisation, collision step and the per-particle
// preparation of the tensor-core projection.
//
// Compiled with -fmad=false: FP64 and FP32 expressions that define the stored
// state are evaluated as separate IEEE operations in source order, so the new
// state is bit-identical to a plain implementation of the same rules.
#include <math.h>
#include <string.h>

#include "df32.cuh"
#include "pc_internal.cuh"

namespace {

constexpr int kMaxCap = 32;

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

__device__ __forceinline__ double minimg_box(double d, double L) {
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

__device__ __forceinline__ float minimgf_box(float d, float L) {
  if (d > 0.5f * L) return d - L;
  if (d < -0.5f * L) return d + L;
  return d;
}

__device__ __forceinline__ double minimg(double d) {
  if (d > 0.5) return d - 1.0;
  if (d < -0.5) return d + 1.0;
  return d;
}

__device__ __forceinline__ void raise_status(unsigned long long* counters, int code) {
  atomicMax(&counters[CNT_STATUS], (unsigned long long)code);
}

__device__ __forceinline__ void cell_coords(int32_t cell, int nc, int c[3]) {
  c[0] = cell % nc;
  c[1] = (cell / nc) % nc;
  c[2] = cell / (nc * nc);
}

// ------------------------------------------------------------------ quantise

__global__ void k_quantize(int64_t n, int nc, const double* __restrict__ x, const double* __restrict__ v,
                           const double* __restrict__ r, const double* __restrict__ m, const double* __restrict__ q,
                           const int32_t* __restrict__ id, int32_t* __restrict__ cell, float* __restrict__ o,
                           float* __restrict__ vf, float* __restrict__ rf, float* __restrict__ mf,
                           float* __restrict__ qf, int32_t* __restrict__ ido) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3];
  for (int a = 0; a < 3; ++a) {
    const double s = x[a * n + i] * (double)nc;
    double fl = floor(s);
    if (fl < 0.0) fl = 0.0;
    if (fl > (double)(nc - 1)) fl = (double)(nc - 1);
    int ci = (int)fl;
    float oo = (float)(s - fl);
    if (oo >= 1.0f) {
      oo = 0.0f;
      ci = ci + 1 == nc ? 0 : ci + 1;
    }
    c[a] = ci;
    o[a * n + i] = oo;
    vf[a * n + i] = (float)v[a * n + i];
  }
  cell[i] = (c[2] * nc + c[1]) * nc + c[0];
  rf[i] = (float)r[i];
  mf[i] = (float)m[i];
  ido[i] = id[i];
  if (qf && q)
    for (int k = 0; k < 4; ++k) qf[k * n + i] = (float)q[k * n + i];
}

// ------------------------------------------------------------------ keys, gather

__global__ void k_keys_f32(int64_t n, int nc, const int32_t* __restrict__ cell, const float* __restrict__ o,
                           const float* __restrict__ v, const float* __restrict__ r, const float* __restrict__ m,
                           int32_t* __restrict__ key, int32_t* __restrict__ slot, int32_t* __restrict__ cnt,
                           unsigned long long* __restrict__ counters) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v2 = 0.0, rr = 0.0;
  if (i < n) {
    const int32_t c = cell[i];
    const int64_t ncell = (int64_t)nc * nc * nc;
    bool ok = c >= 0 && (int64_t)c < ncell;
    for (int a = 0; a < 3; ++a) {
      const float oa = o[a * n + i];
      ok = ok && oa >= 0.0f && oa < 1.0f && isfinite(v[a * n + i]);
    }
    const float ri = r[i], mi = m[i];
    ok = ok && ri > 0.0f && ri < 0.25f && mi > 0.0f && isfinite(mi);
    if (!ok) raise_status(counters, PC_EINVAL);
    const int32_t k = ok ? c : 0;
    key[i] = k;
    slot[i] = atomicAdd(&cnt[k], 1);
    if (ok) {
      // |v|^2 in FP32, rounded up: three roundings (below 2.4e-7 relative) under the
      // factor's 1e-6, so an upper bound of the stored velocity's exact value, which is
      // all the search's reach and filter bounds need (FP64 here would cost a warp 64
      // pipe cycles per instruction on this GPU)
      const float v0 = v[i], v1 = v[n + i], vz = v[2 * n + i];
      v2 = (double)(fmaf(v0, v0, fmaf(v1, v1, vz * vz)) * 1.000001f);
      rr = ri;
    }
  }
  pc_block_max2(&counters[CNT_VMAX2], v2, &counters[CNT_RMAX], rr);
}

__global__ void k_gather_f32(int64_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ cell,
                             const float* __restrict__ o, const float* __restrict__ v, const float* __restrict__ r,
                             const int32_t* __restrict__ id, int32_t* __restrict__ scell, float* __restrict__ so,
                             float* __restrict__ sv, float* __restrict__ sr, int32_t* __restrict__ sid) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t p = perm[k];
  scell[k] = cell[p];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    so[a * n + k] = o[a * n + p];
    sv[a * n + k] = v[a * n + p];
  }
  sr[k] = r[p];
  sid[k] = id[p];
}

// ------------------------------------------------------------------ search

struct SearchF32 {
  int64_t n;
  int nc, cap;
  double dt;
  const int32_t* scell;
  const float *so, *sv, *sr;
  const int32_t* sid;
  const int32_t* start;
  int32_t* cand_j;
  double* cand_t;
  int32_t* ncand;
  int32_t* best;
  unsigned long long* counters;
};

// Smaller positive root of |dx + t dv| = R in cell units (dx the minimum image in a
// box of L cells), with the same operations as the FP64 definition; +inf when the
// pair is not a candidate.
__device__ double contact_time_cells(const double xi[3], const double xj[3], const double vi[3],
                                     const double vj[3], double R, double dt, double L) {
  const double dx0 = minimg_box(xi[0] - xj[0], L);
  const double dx1 = minimg_box(xi[1] - xj[1], L);
  const double dx2 = minimg_box(xi[2] - xj[2], L);
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

// Certified FP32 reject test in cell units. Cell differences are exact integers
// wrapped to the nearest image; offsets are exact FP32, so for candidate pairs
// (a few cells apart) |dxf - dx| <= 2.4e-7 cells per axis. Velocities in cell
// units carry 2^-24 relative error. Same bounds as the FP64 path's filter,
// expressed in cell units.
__device__ __forceinline__ bool filter_cells(const float dxf[3], const float dvc[3], float Rc, float dt,
                                             float vmaxc) {
  const float d2 = dxf[0] * dxf[0] + dxf[1] * dxf[1] + dxf[2] * dxf[2];
  const float v2 = dvc[0] * dvc[0] + dvc[1] * dvc[1] + dvc[2] * dvc[2];
  const float vm = sqrtf(v2);
  const float reach = (Rc + vm * dt) * 1.00001f + 8.0e-7f + 2.5e-7f * vmaxc * dt;
  if (d2 > reach * reach) return false;
  const float bf = dxf[0] * dvc[0] + dxf[1] * dvc[1] + dxf[2] * dvc[2];
  const float bslack = (8.0e-7f + 1.0e-6f * sqrtf(d2)) * (vm + vmaxc);
  return !(bf > bslack);
}

constexpr int kPassCap = 64;  // distance-test passes queued per warp
constexpr int kSurvCap = 64;  // filter survivors queued per warp
constexpr unsigned kFull = 0xffffffffu;

// FP64 root of the pair (k, j) in cell units, with the arguments the step defines.
__device__ __forceinline__ double solve_cells(const SearchF32& A, int64_t k, int64_t j) {
  const int64_t n = A.n;
  const int nc = A.nc;
  const double L = (double)nc;
  int ck[3], cj[3];
  cell_coords(A.scell[k], nc, ck);
  cell_coords(A.scell[j], nc, cj);
  double xi[3], xj[3], vi[3], vj[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xi[a] = (double)ck[a] + (double)A.so[a * n + k];
    xj[a] = (double)cj[a] + (double)A.so[a * n + j];
    vi[a] = (double)A.sv[a * n + k] * L;
    vj[a] = (double)A.sv[a * n + j] * L;
  }
  return contact_time_cells(xi, xj, vi, vj, ((double)A.sr[k] + (double)A.sr[j]) * L, A.dt, L);
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

// Per-warp queues of the contact search in shared memory.
struct SearchQueueF32 {
  float dx[kPassCap], dy[kPassCap], dz[kPassCap];  // offsets of the queued distance-test passes
  int j[kPassCap], own[kPassCap];                  // candidate and owning lane
  int sown[kSurvCap], sj[kSurvCap];                // filter survivors
  double st[kSurvCap];                             // their FP64 roots
};

// Thread per particle (sorted by cell), the warp's lanes in lockstep. The stencil is
// taken row by row; a row's 2 s + 1 cells along x are one contiguous range of the
// sorted arrays, or two where the row wraps. Each candidate first takes a distance
// test against a reach that no pair of this particle exceeds in the filter; the
// passes are queued per warp and, 32 at a time, go through the certified FP32
// filter with one pass per lane. Its survivors are queued again and solved exactly
// in FP64 by the warp's lanes together (on this GPU an FP64 instruction takes a
// warp 64 pipe cycles whatever the number of active lanes); every lane then inserts
// its own roots in [0, dt] into its list sorted by (t, id), which does not depend on
// the order in which they were found. The offsets and tests are the same
// expressions for every pair, so the candidate lists do not depend on the queueing.
__global__ void __launch_bounds__(256, 3) k_search_f32(SearchF32 A) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  const int nc = A.nc;
  const float Lf = (float)nc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  // stencil radius and speed bound from the step's maxima, once per block (FP64 is
  // 1/64 of the FP32 rate on this GPU)
  __shared__ int s_sh;
  __shared__ float vmaxc_sh, rmaxc_sh;
  __shared__ SearchQueueF32 queues[8];
  SearchQueueF32& Q = queues[warp];
  __shared__ int stat_sh[3];  // candidates found, FP64 solves, largest list
  if (threadIdx.x == 0) {
    stat_sh[0] = stat_sh[1] = stat_sh[2] = 0;
    const double L = (double)nc;
    const double v2max = __longlong_as_double((long long)A.counters[CNT_VMAX2]);
    const double rmax = __longlong_as_double((long long)A.counters[CNT_RMAX]);
    const double reach = (2.0 * rmax + 2.0 * sqrt(v2max) * A.dt) * (1.0 + 1e-9) + 1e-12;  // box units
    double sd = floor(reach * L * (1.0 + 1e-9)) + 1.0;
    if (sd > L) sd = L;
    s_sh = (int)sd;
    vmaxc_sh = (float)(sqrt(v2max) * L) * 1.000001f;
    rmaxc_sh = (float)(rmax * L) * 1.000001f;
    if (blockIdx.x == 0) {
      atomicMax(&A.counters[CNT_STENCIL], (unsigned long long)s_sh);
      if (!(reach < 0.5)) raise_status(A.counters, PC_EINVAL);
    }
  }
  __syncthreads();
  const int s = s_sh;
  const float dtf = (float)A.dt * 1.000001f;
  const float vmaxc = vmaxc_sh;
  const bool live = k < n;
  const int64_t kw = (int64_t)blockIdx.x * blockDim.x + 32 * warp;  // the warp's first particle
  int found = 0, solves = 0, cnt = 0;
  double lt[kMaxCap];
  int lj[kMaxCap];
  int ck[3] = {0, 0, 0};
  float ok3[3] = {0.0f, 0.0f, 0.0f}, vk3[3] = {0.0f, 0.0f, 0.0f}, rk = 0.0f, rl2 = -1.0f;
  if (live) {
    cell_coords(A.scell[k], nc, ck);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ok3[a] = A.so[a * n + k];
      vk3[a] = A.sv[a * n + k];
    }
    rk = A.sr[k];
    // A reach no pair of this particle exceeds in filter_cells: (r_k + r_max) nc and
    // (|v_k| nc + vmaxc) for the radius sum and the speed, with margins.
    const float vkc = sqrtf(vk3[0] * vk3[0] + vk3[1] * vk3[1] + vk3[2] * vk3[2]) * Lf * 1.000001f;
    const float rhi = ((rk * Lf + rmaxc_sh) + (vkc + vmaxc) * dtf) * 1.00002f + 8.0e-7f + 2.5e-7f * vmaxc * dtf;
    rl2 = rhi * rhi * 1.0001f;
  }
  int np = 0, ns = 0;  // queued passes and survivors (the same in every lane)

  // the queued survivors' FP64 roots, by the lanes together; each lane then inserts its own
  auto flush_survivors = [&]() {
    for (int e = lane; e < ns; e += 32) {
      Q.st[e] = solve_cells(A, kw + Q.sown[e], Q.sj[e]);
      ++solves;
    }
    __syncwarp();
    for (int e = 0; e < ns; ++e) {
      if (Q.sown[e] != lane) continue;
      const double t = Q.st[e];
      if (t <= A.dt) {
        ++found;
        insert_sorted(lt, lj, cnt, A.cap, t, Q.sj[e], A.sid);
      }
    }
    __syncwarp();
    ns = 0;
  };
  // the certified filter on the first m <= 32 queued passes, one per lane
  auto filter_passes = [&](int m) {
    const int own = lane < m ? Q.own[lane] : lane;
    const float vo0 = __shfl_sync(kFull, vk3[0], own), vo1 = __shfl_sync(kFull, vk3[1], own),
                vo2 = __shfl_sync(kFull, vk3[2], own), ro = __shfl_sync(kFull, rk, own);
    bool keep = false;
    int j = 0;
    if (lane < m) {
      j = Q.j[lane];
      const float dxf[3] = {Q.dx[lane], Q.dy[lane], Q.dz[lane]};
      const float dvc[3] = {(vo0 - A.sv[j]) * Lf, (vo1 - A.sv[n + j]) * Lf, (vo2 - A.sv[2 * n + j]) * Lf};
      keep = filter_cells(dxf, dvc, (ro + A.sr[j]) * Lf, dtf, vmaxc);
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
  // offsets below s + 1 <= nc / 2 are their own minimum image
  const bool need_box = 2 * (s + 1) > nc;
  // per-axis bases of the candidate arrays and a 32-bit own index for the inner loop
  const int32_t* __restrict__ scell_p = A.scell;
  const float* __restrict__ so0 = A.so;
  const float* __restrict__ so1 = A.so + n;
  const float* __restrict__ so2 = A.so + 2 * n;
  const int k32 = live ? (int)k : -1;
  for (int oz = 0; oz < cnt_ax; ++oz) {
    for (int oy = 0; oy < cnt_ax; ++oy) {
      int b1 = 0, e1 = 0, b2 = 0, e2 = 0, rowck = 0;
      float dyf = 0.0f, dzf = 0.0f;
      if (live) {
        const int zc = full ? oz : wrapi(ck[2] - s + oz, nc);
        const int yc = full ? oy : wrapi(ck[1] - s + oy, nc);
        int dyi = ck[1] - yc, dzi = ck[2] - zc;
        if (2 * dyi > nc) dyi -= nc;
        else if (2 * dyi < -nc) dyi += nc;
        if (2 * dzi > nc) dzi -= nc;
        else if (2 * dzi < -nc) dzi += nc;
        dyf = (float)dyi;
        dzf = (float)dzi;
        const int row = (zc * nc + yc) * nc;
        rowck = row + ck[0];
        const int xl = ck[0] - s, xh = ck[0] + s;
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
          int di = rowck - scell_p[j];
          if (2 * di > nc) di -= nc;
          else if (2 * di < -nc) di += nc;
          dx = (float)di + (ok3[0] - so0[j]);
          dy = dyf + (ok3[1] - so1[j]);
          dz = dzf + (ok3[2] - so2[j]);
          if (need_box) {
            dx = minimgf_box(dx, Lf);
            dy = minimgf_box(dy, Lf);
            dz = minimgf_box(dz, Lf);
          }
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

// ------------------------------------------------------------------ respond

struct RespondF32 {
  int64_t n;
  int nc;
  double dt, e;
  const int32_t* scell;
  const float *so, *sv, *sr;
  const int32_t* sid;
  const int32_t* partner;
  const double* tcoll;
  const int32_t* perm;
  const float* m_in;
  const float* q_in;
  int32_t* cell_out;
  float *o_out, *v_out, *r_out, *m_out, *q_out;
  int32_t* id_out;
  int32_t* list;                    // [n]: sorted indices of the colliding particles
  unsigned long long* counters;     // CNT_RESP counts them
};

// Free flight of one axis: o' = o + float(dt nc) v in FP32 with a carry into the
// neighbouring cell (periodic).
__device__ __forceinline__ float advance_free_axis(float o, float va, float dtn, int nc, int* c) {
  float on = o + dtn * va;
  if (on >= 1.0f) {
    on = on - 1.0f;
    *c = *c + 1 == nc ? 0 : *c + 1;
  } else if (on < 0.0f) {
    const float up = on + 1.0f;
    if (up == 1.0f) {
      on = 0.0f;
    } else {
      on = up;
      *c = *c == 0 ? nc - 1 : *c - 1;
    }
  }
  return on;
}

// Response of particle i of a colliding pair (i, j) at contact time t, in cell
// units: FP64 response from the stored values, new position wrapped into [0, nc)
// and stored as floor + FP32 offset (carried when it rounds to 1), velocity
// rounded to FP32. c[] holds i's cell on entry and its new cell on exit.
__device__ __forceinline__ void respond_pair_f32(int c[3], const int cj[3], const float oi[3], const float oj[3],
                                                 const float vi[3], const float vj[3], float mi_f, float mj_f,
                                                 double t, double dt, double e, int nc, float oo[3], float vo[3]) {
  const double L = (double)nc;
  double xi[3], dx[3], dvc[3], dv[3], s3[3], nr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xi[a] = (double)c[a] + (double)oi[a];
    const double xj = (double)cj[a] + (double)oj[a];
    dx[a] = minimg_box(xi[a] - xj, L);
    dvc[a] = (double)vi[a] * L - (double)vj[a] * L;
    dv[a] = (double)vi[a] - (double)vj[a];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) s3[a] = dx[a] + t * dvc[a];
  const double sl = sqrt((s3[0] * s3[0] + s3[1] * s3[1]) + s3[2] * s3[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) nr[a] = -s3[a] / sl;
  const double vrn = (dv[0] * nr[0] + dv[1] * nr[1]) + dv[2] * nr[2];
  const double mi = (double)mi_f, mj = (double)mj_f;
  const double mr = (mi * mj) / (mi + mj);
  const double J = -mr * (1.0 + e) * vrn;
  const double gi = J / mi;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double vold = (double)vi[a];
    const double vnew = vold + gi * nr[a];
    double y = (xi[a] + t * (vold * L)) + (dt - t) * (vnew * L);
    if (y < 0.0) y += L;
    else if (y >= L) y -= L;
    double fl = floor(y);
    if (fl < 0.0) fl = 0.0;
    if (fl > (double)(nc - 1)) fl = (double)(nc - 1);
    int cq = (int)fl;
    float oq = (float)(y - fl);
    if (oq >= 1.0f) {
      oq = 0.0f;
      cq = cq + 1 == nc ? 0 : cq + 1;
    }
    c[a] = cq;
    oo[a] = oq;
    vo[a] = (float)vnew;
  }
}

// Free particles: advance_free_axis on each axis. Colliding particles go to a list
// (slots once per warp) and k_respond_pairs_f32 computes their FP64 responses with
// every lane of a warp busy: on this GPU an FP64 instruction takes a warp 64 pipe
// cycles whatever the number of active lanes, and a block's few colliding lanes
// would otherwise hold it for the whole response.
__global__ void __launch_bounds__(256) k_respond_f32(RespondF32 R) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = R.n;
  const int nc = R.nc;
  const int lane = threadIdx.x & 31;
  bool col = false;
  if (k < n) {
    const int64_t p = R.perm[k];
    const int32_t j = R.partner[k];
    const float mi_f = R.m_in[p];
    if (j < 0) {
      int c[3];
      cell_coords(R.scell[k], nc, c);
      const float dtn = (float)(R.dt * (double)nc);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float v = R.sv[a * n + k];
        R.o_out[a * n + k] = advance_free_axis(R.so[a * n + k], v, dtn, nc, &c[a]);
        R.v_out[a * n + k] = v;
      }
      R.cell_out[k] = (c[2] * nc + c[1]) * nc + c[0];
    } else {
      col = true;
    }
    R.r_out[k] = R.sr[k];
    R.m_out[k] = mi_f;
    R.id_out[k] = R.sid[k];
    if (R.q_out)
      for (int q = 0; q < 4; ++q) R.q_out[q * n + k] = R.q_in[q * n + p];
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

// Responses of the listed colliding particles (respond_pair_f32 from each particle's
// own side), grid-stride over the list.
__global__ void __launch_bounds__(256) k_respond_pairs_f32(RespondF32 R) {
  const int64_t cnt = (int64_t)R.counters[CNT_RESP];
  const int64_t n = R.n;
  const int nc = R.nc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kk = R.list[i];
    const int32_t j = R.partner[kk];
    int c[3], cj[3];
    cell_coords(R.scell[kk], nc, c);
    cell_coords(R.scell[j], nc, cj);
    const float oi[3] = {R.so[kk], R.so[n + kk], R.so[2 * n + kk]}, oj[3] = {R.so[j], R.so[n + j], R.so[2 * n + j]};
    const float vi[3] = {R.sv[kk], R.sv[n + kk], R.sv[2 * n + kk]}, vj[3] = {R.sv[j], R.sv[n + j], R.sv[2 * n + j]};
    float oo[3], vo[3];
    respond_pair_f32(c, cj, oi, oj, vi, vj, R.m_in[R.perm[kk]], R.m_in[R.perm[j]], R.tcoll[kk], R.dt, R.e, nc, oo,
                     vo);
    R.cell_out[kk] = (c[2] * nc + c[1]) * nc + c[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R.o_out[a * n + kk] = oo[a];
      R.v_out[a * n + kk] = vo[a];
    }
  }
}

// ------------------------------------------------------------------ projection prep

// Element of a cell-relative coordinate: floor((c + o) ne / nc) in df32, the same
// function for the binning and for the factors.
__device__ __forceinline__ int elem_of(int c, float o, f2 rnn, int ne, float* t) {
  const f2 xc = two_sum((float)c, o);  // exact
  const f2 u = df_mul(xc, rnn);
  float e = floorf(u.h);
  if (u.h == e && u.l < 0.0f) e -= 1.0f;
  int ei = (int)e;
  float tt = (u.h - e) + u.l;
  if (ei < 0) {
    ei = 0;
    tt = 0.0f;
  }
  if (ei > ne - 1) {
    ei = ne - 1;
    tt = 1.0f;
  }
  *t = tt;
  return ei;
}

__global__ void k_elem_keys_f32(int64_t n, int nc, int ne, f2 rnn, const int32_t* __restrict__ cell,
                                const float* __restrict__ o, int32_t* __restrict__ key, int32_t* __restrict__ slot,
                                int32_t* __restrict__ cnt, unsigned long long* __restrict__ counters) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3];
  const int32_t cl = cell[i];
  if (!(cl >= 0 && (int64_t)cl < (int64_t)nc * nc * nc)) raise_status(counters, PC_EINVAL);
  cell_coords(cl < 0 ? 0 : cl, nc, c);
  int e[3];
  float t;
  for (int a = 0; a < 3; ++a) {
    const float oa = o[a * n + i];
    if (!(oa >= 0.0f && oa < 1.0f)) raise_status(counters, PC_EINVAL);
    e[a] = elem_of(min(max(c[a], 0), nc - 1), oa, rnn, ne, &t);
  }
  const int k = (e[2] * ne + e[1]) * ne + e[0];
  key[i] = k;
  slot[i] = atomicAdd(&cnt[k], 1);
}

// 2^x by the hardware approximation, the one the tensor-core deposit evaluates its
// factors with, so that 1/Z normalises exactly those factors.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct PrepF32 {
  int64_t n;
  int nc, ne, n1, rho, win;
  f2 rnn;           // ne / nc
  float rce;        // cutoff in element units
  float c2l;        // h^2 / (2 sigma^2) log2(e)
  double h, rc;
  float s[64];      // window node offsets o + (eta_i + 1)/2 in element units
  float wq[64];     // Gauss weight of each window node (w % n1)
  double eta[16];
  const int32_t* perm;
  const int32_t* cell;
  const float* o;
  const float* q;
  float4* rec;      // [n][4]
};

// Per particle (sorted by element): position t_a in its own element's units, the
// inside-cutoff mask of the 3 (2 rho + 1) n1 window nodes, 1/Z_a with
// Z_a = sum over inside nodes of w_i exp(-(delta h)^2/(2 sigma^2)), q, and per axis
// which of the 2 rho + 1 window elements hold an inside node. A node whose FP32 distance is within 1e-4 relative of the cutoff is decided in
// FP64 on the stored position x = (c + o)/nc with the plain definition.
__global__ void __launch_bounds__(128) k_proj_prep_f32(PrepF32 P) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = P.n;
  if (k >= n) return;
  const int64_t p = P.perm[k];
  int c[3];
  cell_coords(P.cell[p], P.nc, c);
  float t3[3], iz[3];
  unsigned mask[3];
  for (int a = 0; a < 3; ++a) {
    const float oa = P.o[a * n + p];
    float t;
    const int ea = elem_of(c[a], oa, P.rnn, P.ne, &t);
    float Z = 0.0f;
    unsigned mk = 0u;
    for (int w = 0; w < P.win; ++w) {
      const float d = P.s[w] - t;
      const float ad = fabsf(d);
      bool inside;
      if (fabsf(ad - P.rce) > 1e-4f * P.rce) {
        inside = ad < P.rce;
      } else {
        const int i = w % P.n1, off = w / P.n1 - P.rho;
        const int ge = wrapi(ea + off, P.ne);
        const double x = ((double)c[a] + (double)oa) / (double)P.nc;
        const double X = ((double)ge + 0.5 * (P.eta[i] + 1.0)) * P.h;
        inside = fabs(minimg(X - x)) <= P.rc;
      }
      if (inside) {
        mk |= 1u << w;
        Z += P.wq[w] * ex2_approx(-(d * d) * P.c2l);
      }
    }
    t3[a] = t;
    iz[a] = Z > 0.0f ? 1.0f / Z : 0.0f;
    mask[a] = mk;
  }
  float4* rp = P.rec + 4 * k;
  const float q0 = P.q[p], q1 = P.q[n + p], q2 = P.q[2 * n + p], q3 = P.q[3 * n + p];
  rp[0] = make_float4(t3[0], t3[1], t3[2], iz[0]);
  rp[1] = make_float4(iz[1], iz[2], q0, q1);
  rp[2] = make_float4(q2, q3, __uint_as_float(mask[0]), __uint_as_float(mask[1]));
  // reach bits: bit 8 a + wo set when window block wo of axis a holds an inside node
  unsigned reach = 0u;
  const unsigned nmask = (1u << P.n1) - 1u;
  for (int a = 0; a < 3; ++a)
    for (int wo = 0; wo < 2 * P.rho + 1; ++wo)
      if ((mask[a] >> (wo * P.n1)) & nmask) reach |= 1u << (8 * a + wo);
  rp[3] = make_float4(__uint_as_float(mask[2]), __uint_as_float(reach), 0.0f, 0.0f);
}

// ------------------------------------------------------------------ FP32 rollouts

struct ReplayF32 {
  int64_t n;
  int nc;
  double dt, e;
  const int32_t* cell;
  const float *o, *v, *r, *m, *q;
  const int32_t* id;
  const int32_t* partner;
  int32_t* cell_out;
  float *o_out, *v_out, *r_out, *m_out, *q_out;
  int32_t* id_out;
  unsigned long long* counters;
};

// Contact time of the pair (i, j) from i's side, with the arguments the search
// forms: exact FP64 positions in cell units, v nc, (r_i + r_j) nc.
__device__ __forceinline__ double pair_time_cells(const int ci[3], const int cj[3], const float oi[3],
                                                  const float oj[3], const float vi[3], const float vj[3], float ri,
                                                  float rj, double dt, int nc) {
  const double L = (double)nc;
  double xi[3], xj[3], vci[3], vcj[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xi[a] = (double)ci[a] + (double)oi[a];
    xj[a] = (double)cj[a] + (double)oj[a];
    vci[a] = (double)vi[a] * L;
    vcj[a] = (double)vj[a] * L;
  }
  return contact_time_cells(xi, xj, vci, vcj, ((double)ri + (double)rj) * L, dt, L);
}

// One mixed step with a given pair set, in the order of the arrays (partner[i] =
// index of i's partner, or -1): the contact time of the search, then the same
// free flight and response as k_respond_f32, hence bit-identical to
// pc_collide_f32 for the pair set it chose.
// The replayed pair step of particle i (partner j >= 0); a pair without a root in
// [0, dt] is recorded as PC_EREPLAY and flies free.
__device__ __forceinline__ void replay_pair_f32(const ReplayF32& R, int64_t i, int32_t j) {
  const int64_t n = R.n;
  const int nc = R.nc;
  int c[3];
  cell_coords(R.cell[i], nc, c);
  const float oi[3] = {R.o[i], R.o[n + i], R.o[2 * n + i]};
  const float vi[3] = {R.v[i], R.v[n + i], R.v[2 * n + i]};
  float oo[3], vo[3];
  int cj[3];
  cell_coords(R.cell[j], nc, cj);
  const float oj[3] = {R.o[j], R.o[n + j], R.o[2 * n + j]};
  const float vj[3] = {R.v[j], R.v[n + j], R.v[2 * n + j]};
  const double t = pair_time_cells(c, cj, oi, oj, vi, vj, R.r[i], R.r[j], R.dt, nc);
  if (t <= R.dt) {
    respond_pair_f32(c, cj, oi, oj, vi, vj, R.m[i], R.m[j], t, R.dt, R.e, nc, oo, vo);
  } else {
    raise_status(R.counters, PC_EREPLAY);
    const float dtn = (float)(R.dt * (double)nc);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      vo[a] = vi[a];
      oo[a] = advance_free_axis(oi[a], vi[a], dtn, nc, &c[a]);
    }
  }
  R.cell_out[i] = (c[2] * nc + c[1]) * nc + c[0];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R.o_out[a * n + i] = oo[a];
    R.v_out[a * n + i] = vo[a];
  }
}

// One mixed step with a given pair set, in the order of the arrays (partner[i] =
// index of i's partner, or -1): the contact time of the search, then the same
// free flight and response as k_respond_f32, hence bit-identical to
// pc_collide_f32 for the pair set it chose. The block's colliding particles are
// replayed by its first threads together, as in k_respond_f32.
__global__ void __launch_bounds__(256) k_replay_f32(ReplayF32 R) {
  __shared__ int q_cnt;
  __shared__ int q_i[256];
  if (threadIdx.x == 0) q_cnt = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = R.n;
  const int nc = R.nc;
  if (i < n) {
    if (R.partner[i] < 0) {
      int c[3];
      cell_coords(R.cell[i], nc, c);
      const float dtn = (float)(R.dt * (double)nc);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float vi = R.v[a * n + i];
        R.o_out[a * n + i] = advance_free_axis(R.o[a * n + i], vi, dtn, nc, &c[a]);
        R.v_out[a * n + i] = vi;
      }
      R.cell_out[i] = (c[2] * nc + c[1]) * nc + c[0];
    } else {
      q_i[atomicAdd(&q_cnt, 1)] = threadIdx.x;
    }
    if (R.r_out) R.r_out[i] = R.r[i];
    if (R.m_out) R.m_out[i] = R.m[i];
    if (R.id_out) R.id_out[i] = R.id[i];
    if (R.q_out)
      for (int q = 0; q < 4; ++q) R.q_out[q * n + i] = R.q[q * n + i];
  }
  __syncthreads();
  const int nq = q_cnt;
  for (int e = threadIdx.x; e < nq; e += blockDim.x) {
    const int64_t ii = (int64_t)blockIdx.x * blockDim.x + q_i[e];
    replay_pair_f32(R, ii, R.partner[ii]);
  }
}

struct AdjF32 {
  int64_t n;
  int nc;
  double dt, e;
  const int32_t* cell;
  const float *o, *v, *r, *m;
  const int32_t* partner;
  const float *gxo, *gvo;
  float *gxi, *gvi;
  unsigned long long* counters;
};

// Vector-Jacobian product of the mixed step in FP32, physical units, the pair set
// fixed and the storage rounding taken as the identity. The contact time is the
// FP64 root of the forward step (the value the step used); every derivative is
// evaluated in FP32: t through |dx + t dv| = R (implicit function theorem),
// n = -s/|s|, J = -m_r (1+e) dv.n, v' = v + (J/m) n, x' = x + t v + (dt - t) v'.
__device__ __forceinline__ void adjoint_pair_f32(const AdjF32& A, int64_t i, int32_t j) {
  const int64_t n = A.n;
  const float dtf = (float)A.dt;
  const int nc = A.nc;
  int ci[3], cj[3];
  cell_coords(A.cell[i], nc, ci);
  cell_coords(A.cell[j], nc, cj);
  const float oi[3] = {A.o[i], A.o[n + i], A.o[2 * n + i]}, oj[3] = {A.o[j], A.o[n + j], A.o[2 * n + j]};
  const float vi[3] = {A.v[i], A.v[n + i], A.v[2 * n + i]}, vj[3] = {A.v[j], A.v[n + j], A.v[2 * n + j]};
  const double t64 = pair_time_cells(ci, cj, oi, oj, vi, vj, A.r[i], A.r[j], A.dt, nc);
  if (!(t64 <= A.dt)) {
    raise_status(A.counters, PC_EREPLAY);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      A.gxi[a * n + i] = 0.0f;
      A.gvi[a * n + i] = 0.0f;
    }
    return;
  }
  const float t = (float)t64, inv_nc = 1.0f / (float)nc, Lf = (float)nc;
  const float mi = A.m[i], mj = A.m[j];
  float dx[3], dv[3], s[3], nr[3], vin[3], vjn[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // cell difference wrapped to the nearest image, then the exact offset difference
    int di = ci[a] - cj[a];
    if (2 * di > nc) di -= nc;
    else if (2 * di < -nc) di += nc;
    dx[a] = minimgf_box((float)di + (oi[a] - oj[a]), Lf) * inv_nc;
    dv[a] = vi[a] - vj[a];
    s[a] = dx[a] + t * dv[a];
  }
  const float sl = sqrtf((s[0] * s[0] + s[1] * s[1]) + s[2] * s[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) nr[a] = -s[a] / sl;
  const float vrn = (dv[0] * nr[0] + dv[1] * nr[1]) + dv[2] * nr[2];
  const float mr = (mi * mj) / (mi + mj);
  const float J = -mr * (1.0f + (float)A.e) * vrn;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    vin[a] = vi[a] + (J / mi) * nr[a];
    vjn[a] = vj[a] - (J / mj) * nr[a];
  }
  float Vit[3], Vjt[3], gn[3] = {0.0f, 0.0f, 0.0f}, gdv[3] = {0.0f, 0.0f, 0.0f}, gdx[3] = {0.0f, 0.0f, 0.0f},
        gvi_own[3];
  float gt = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float Xi = A.gxo[a * n + i], Xj = A.gxo[a * n + j];
    gvi_own[a] = t * Xi;
    Vit[a] = A.gvo[a * n + i] + (dtf - t) * Xi;
    Vjt[a] = A.gvo[a * n + j] + (dtf - t) * Xj;
    gt += Xi * (vi[a] - vin[a]) + Xj * (vj[a] - vjn[a]);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gvi_own[a] += Vit[a];
    gn[a] += (J / mi) * Vit[a] - (J / mj) * Vjt[a];
  }
  const float gJ = ((Vit[0] * nr[0] + Vit[1] * nr[1]) + Vit[2] * nr[2]) / mi -
                   ((Vjt[0] * nr[0] + Vjt[1] * nr[1]) + Vjt[2] * nr[2]) / mj;
  const float gvrn = -mr * (1.0f + (float)A.e) * gJ;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gdv[a] += gvrn * nr[a];
    gn[a] += gvrn * dv[a];
  }
  const float nh[3] = {s[0] / sl, s[1] / sl, s[2] / sl};
  const float pg = (nh[0] * gn[0] + nh[1] * gn[1]) + nh[2] * gn[2];
  float gs[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) gs[a] = -(gn[a] - nh[a] * pg) / sl;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gdx[a] += gs[a];
    gdv[a] += t * gs[a];
  }
  gt += (gs[0] * dv[0] + gs[1] * dv[1]) + gs[2] * dv[2];
  const float sdv = (s[0] * dv[0] + s[1] * dv[1]) + s[2] * dv[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gdx[a] += gt * (-s[a] / sdv);
    gdv[a] += gt * (-t * s[a] / sdv);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    A.gxi[a * n + i] = A.gxo[a * n + i] + gdx[a];
    A.gvi[a * n + i] = gvi_own[a] + gdv[a];
  }
}

// One thread per particle for the free ones; the block's colliding particles are
// swept by its first threads together, as in k_replay_f32.
__global__ void __launch_bounds__(256) k_collide_adjoint_f32(AdjF32 A) {
  __shared__ int q_cnt;
  __shared__ int q_i[256];
  if (threadIdx.x == 0) q_cnt = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  const float dtf = (float)A.dt;
  if (i < n) {
    if (A.partner[i] < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float X = A.gxo[a * n + i];
        A.gxi[a * n + i] = X;
        A.gvi[a * n + i] = A.gvo[a * n + i] + dtf * X;
      }
    } else {
      q_i[atomicAdd(&q_cnt, 1)] = threadIdx.x;
    }
  }
  __syncthreads();
  const int nq = q_cnt;
  for (int e = threadIdx.x; e < nq; e += blockDim.x) {
    const int64_t ii = (int64_t)blockIdx.x * blockDim.x + q_i[e];
    adjoint_pair_f32(A, ii, A.partner[ii]);
  }
}

struct ProjAdjF32 {
  int64_t n;
  int nc, ne, n1, rho, win;
  f2 rnn;             // ne / nc
  float rce, c2l;     // cutoff in element units; h^2 / (2 sigma^2) log2(e)
  float scale;        // (2/h)^3
  float hs2;          // h / sigma^2
  double h, rc;
  float s[64];        // window node offsets in element units
  float wq[16];
  double eta[16];
  const int32_t* cell;
  const float *o, *q, *G;
  float *gq, *gx;
};

// Vector-Jacobian product of pc_project_f32 in FP32, one warp per particle: the
// window factors and the inside-cutoff decisions of the forward preparation, Z_a,
// the weighted mean offsets mu_a, then a sweep over the support box reading G:
//   gq_c = (2/h)^3 sum_g G_gc khat, gx_a = (2/h)^3 h / sigma^2 sum_g a_g khat (d_a - mu_a),
// with d in element units, a_g = sum_c G_gc q_c and khat = kx ky kz / (Zx Zy Zz).
__global__ void __launch_bounds__(128) k_project_adjoint_f32(ProjAdjF32 A) {
  __shared__ float kf[4][3][64];
  __shared__ float dd[4][3][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * 4 + warp;
  if (p >= A.n) return;
  const int64_t n = A.n;
  const int n1 = A.n1, ne = A.ne, nc = A.nc, win = A.win, nodes = n1 * n1 * n1;
  int c[3], ea[3];
  float t3[3];
  cell_coords(A.cell[p], nc, c);
#pragma unroll
  for (int a = 0; a < 3; ++a) ea[a] = elem_of(c[a], A.o[a * n + p], A.rnn, ne, &t3[a]);
  for (int u = lane; u < 3 * win; u += 32) {
    const int a = u / win, w = u - a * win;
    const float d = A.s[w] - t3[a];
    const float ad = fabsf(d);
    bool inside;
    if (fabsf(ad - A.rce) > 1e-4f * A.rce) {
      inside = ad < A.rce;
    } else {
      const int i = w % n1, off = w / n1 - A.rho;
      const int ge = wrapi(ea[a] + off, ne);
      const double x = ((double)c[a] + (double)A.o[a * n + p]) / (double)nc;
      const double X = ((double)ge + 0.5 * (A.eta[i] + 1.0)) * A.h;
      inside = fabs(minimg(X - x)) <= A.rc;
    }
    kf[warp][a][w] = inside ? exp2f(-(d * d) * A.c2l) : 0.0f;
    dd[warp][a][w] = d;
  }
  __syncwarp();
  float Z[3], mu[3];
  int lo[3], cnt[3];
  for (int a = 0; a < 3; ++a) {
    float z = 0.0f, z1 = 0.0f;
    int l = -1, hgh = -2;
    for (int w = 0; w < win; ++w) {
      const float k = kf[warp][a][w];
      if (k != 0.0f) {
        if (l < 0) l = w;
        hgh = w;
      }
      z += A.wq[w % n1] * k;
      z1 += A.wq[w % n1] * k * dd[warp][a][w];
    }
    Z[a] = z;
    mu[a] = z > 0.0f ? z1 / z : 0.0f;
    lo[a] = l < 0 ? 0 : l;
    cnt[a] = hgh >= l ? hgh - l + 1 : 0;
  }
  const float q0 = A.q[p], q1 = A.q[n + p], q2 = A.q[2 * n + p], q3 = A.q[3 * n + p];
  float aq[4] = {0.0f, 0.0f, 0.0f, 0.0f}, ax[3] = {0.0f, 0.0f, 0.0f};
  const int nbox = cnt[0] * cnt[1] * cnt[2];
  for (int u = lane; u < nbox; u += 32) {
    const int wx = lo[0] + u % cnt[0];
    const int wy = lo[1] + (u / cnt[0]) % cnt[1];
    const int wz = lo[2] + u / (cnt[0] * cnt[1]);
    const float kx = kf[warp][0][wx], ky = kf[warp][1][wy], kz = kf[warp][2][wz];
    if (kx == 0.0f || ky == 0.0f || kz == 0.0f) continue;
    const int gex = wrapi(ea[0] + wx / n1 - A.rho, ne), gey = wrapi(ea[1] + wy / n1 - A.rho, ne),
              gez = wrapi(ea[2] + wz / n1 - A.rho, ne);
    const int64_t e = ((int64_t)gez * ne + gey) * ne + gex;
    const int64_t g = e * 4 * nodes + ((int64_t)(wz % n1) * n1 + (wy % n1)) * n1 + (wx % n1);
    const float G0 = A.G[g], G1 = A.G[g + nodes], G2 = A.G[g + 2 * nodes], G3 = A.G[g + 3 * nodes];
    const float kh = (kx * ky) * kz;
    aq[0] += G0 * kh;
    aq[1] += G1 * kh;
    aq[2] += G2 * kh;
    aq[3] += G3 * kh;
    const float akh = (((G0 * q0 + G1 * q1) + G2 * q2) + G3 * q3) * kh;
    ax[0] += akh * (dd[warp][0][wx] - mu[0]);
    ax[1] += akh * (dd[warp][1][wy] - mu[1]);
    ax[2] += akh * (dd[warp][2][wz] - mu[2]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    for (int k = 0; k < 4; ++k) aq[k] += __shfl_xor_sync(0xffffffffu, aq[k], o);
    for (int a = 0; a < 3; ++a) ax[a] += __shfl_xor_sync(0xffffffffu, ax[a], o);
  }
  if (lane == 0) {
    const float zz = (Z[0] * Z[1]) * Z[2];
    const float f = zz > 0.0f ? A.scale / zz : 0.0f;
    for (int k = 0; k < 4; ++k) A.gq[k * n + p] = aq[k] * f;
    for (int a = 0; a < 3; ++a) A.gx[a * n + p] = ax[a] * f * A.hs2;
  }
}

}  // namespace

pc_status pc_quantize_impl(pc_ctx* ctx, const pc_particles* in, pc_particles_f32* out) {
  const int64_t n = in->n;
  if (n == 0) return PC_OK;
  k_quantize<<<pc_blocks(n, 256), 256, 0, ctx->stream>>>(n, ctx->nc, in->x, in->v, in->r, in->m, in->q, in->id,
                                                          out->cell, out->o, out->v, out->r, out->m, out->q, out->id);
  ctx->launches += 1;
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_quantize: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}

pc_status pc_collide_f32_impl(pc_ctx* ctx, const pc_particles_f32* in, pc_particles_f32* out, double dt) {
  const int64_t n = in->n;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned long long) * CNT_N, st);
  if (e == cudaSuccess && n == 0) return PC_OK;
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->cnt, 0, sizeof(int32_t) * (size_t)ctx->ncell, st);
  if (e != cudaSuccess) goto fail;
  {
    const int tb = pc_phase_begin(ctx, PC_PH_BIN);
    k_keys_f32<<<pc_blocks(n, 256), 256, 0, st>>>(n, ctx->nc, in->cell, in->o, in->v, in->r, in->m, ctx->key,
                                                   ctx->slot, ctx->cnt, ctx->counters);
    ctx->launches += 1;
    e = pc_bin_finish(n, ctx->ncell, ctx->key, ctx->slot, in->id, ctx->cnt, ctx->start, ctx->blocksums, ctx->perm, st,
                      &ctx->launches);
    pc_phase_end(ctx, tb);
  }
  if (e != cudaSuccess) goto fail;
  {
    const int tg = pc_phase_begin(ctx, PC_PH_GATHER);
    k_gather_f32<<<pc_blocks(n, 256), 256, 0, st>>>(n, ctx->perm, in->cell, in->o, in->v, in->r, in->id,
                                                     ctx->scell, ctx->sxf, ctx->svf, ctx->srf, ctx->sid);
    ctx->launches += 1;
    pc_phase_end(ctx, tg);
  }
  {
    SearchF32 A;
    A.n = n;
    A.nc = ctx->nc;
    A.cap = ctx->cap;
    A.dt = dt;
    A.scell = ctx->scell;
    A.so = ctx->sxf;
    A.sv = ctx->svf;
    A.sr = ctx->srf;
    A.sid = ctx->sid;
    A.start = ctx->start;
    A.cand_j = ctx->cand_j;
    A.cand_t = ctx->cand_t;
    A.ncand = ctx->ncand;
    A.best = ctx->best;
    A.counters = ctx->counters;
    const int ts = pc_phase_begin(ctx, PC_PH_SEARCH);
    k_search_f32<<<pc_blocks(n, 256), 256, 0, st>>>(A);
    ctx->launches += 1;
    pc_phase_end(ctx, ts);
  }
  e = pc_match_launch(ctx, n);
  if (e != cudaSuccess) goto fail;
  {
    RespondF32 R;
    R.n = n;
    R.nc = ctx->nc;
    R.dt = dt;
    R.e = ctx->cfg.restitution;
    R.scell = ctx->scell;
    R.so = ctx->sxf;
    R.sv = ctx->svf;
    R.sr = ctx->srf;
    R.sid = ctx->sid;
    R.partner = ctx->partner;
    R.tcoll = ctx->tcoll;
    R.perm = ctx->perm;
    R.m_in = in->m;
    R.q_in = in->q;
    R.cell_out = out->cell;
    R.o_out = out->o;
    R.v_out = out->v;
    R.r_out = out->r;
    R.m_out = out->m;
    R.q_out = in->q ? out->q : nullptr;
    R.id_out = out->id;
    R.list = ctx->work;  // the matching's work list is spent by now
    R.counters = ctx->counters;
    const int tr = pc_phase_begin(ctx, PC_PH_RESPOND);
    k_respond_f32<<<pc_blocks(n, 256), 256, 0, st>>>(R);
    const int gp = pc_blocks(n, 256) < 4096 ? pc_blocks(n, 256) : 4096;
    k_respond_pairs_f32<<<gp, 256, 0, st>>>(R);
    ctx->launches += 2;
    pc_phase_end(ctx, tr);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
fail:
  snprintf(ctx->err, sizeof(ctx->err), "pc_collide_f32: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}

pc_status pc_project_f32_impl(pc_ctx* ctx, const pc_particles_f32* p, float* field, int tc_type) {
  const int64_t n = p->n;
  cudaStream_t st = ctx->stream;
  const int ne = ctx->cfg.ne;
  const int64_t nel = (int64_t)ne * ne * ne;
  const double rnn = (double)ne / (double)ctx->nc;
  const f2 rnnf = {(float)rnn, (float)(rnn - (double)(float)rnn)};
  cudaError_t e = cudaMemsetAsync(ctx->cnt, 0, sizeof(int32_t) * (size_t)nel, st);
  if (e != cudaSuccess) goto fail;
  {
    const int tb = pc_phase_begin(ctx, PC_PH_PBIN);
    if (n > 0) {
      k_elem_keys_f32<<<pc_blocks(n, 256), 256, 0, st>>>(n, ctx->nc, ne, rnnf, p->cell, p->o, ctx->key, ctx->slot,
                                                          ctx->cnt, ctx->counters);
      ctx->launches += 1;
    }
    e = pc_bin_finish(n, nel, ctx->key, ctx->slot, p->id, ctx->cnt, ctx->start, ctx->blocksums, ctx->perm, st,
                      &ctx->launches);
    pc_phase_end(ctx, tb);
  }
  if (e != cudaSuccess) goto fail;
  if (n > 0) {
    PrepF32 P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.nc = ctx->nc;
    P.ne = ne;
    P.n1 = ctx->n1;
    P.rho = ctx->rho;
    P.win = ctx->win;
    P.rnn = rnnf;
    P.h = ctx->h;
    P.rc = ctx->cfg.cutoff_sigmas * ctx->cfg.sigma;
    P.rce = (float)(P.rc * ne);
    P.c2l = (float)(ctx->h * ctx->h / (2.0 * ctx->cfg.sigma * ctx->cfg.sigma) * 1.4426950408889634);
    for (int w = 0; w < ctx->win; ++w)
      P.s[w] = (float)((double)(w / ctx->n1 - ctx->rho) + 0.5 * (ctx->eta[w % ctx->n1] + 1.0));
    for (int w = 0; w < ctx->win; ++w) P.wq[w] = (float)ctx->w[w % ctx->n1];
    for (int i = 0; i < ctx->n1; ++i) P.eta[i] = ctx->eta[i];
    P.perm = ctx->perm;
    P.cell = p->cell;
    P.o = p->o;
    P.q = p->q;
    P.rec = (float4*)ctx->fac;
    const int tf = pc_phase_begin(ctx, PC_PH_FACTORS);
    k_proj_prep_f32<<<pc_blocks(n, 128), 128, 0, st>>>(P);
    ctx->launches += 1;
    pc_phase_end(ctx, tf);
  }
  {
    TcDepositArgs T;
    memset(&T, 0, sizeof(T));
    T.n = n;
    T.ne = ne;
    T.n1 = ctx->n1;
    T.rho = ctx->rho;
    T.tc_type = tc_type;
    T.c2l = (float)(ctx->h * ctx->h / (2.0 * ctx->cfg.sigma * ctx->cfg.sigma) * 1.4426950408889634);
    T.rce = (float)(ctx->cfg.cutoff_sigmas * ctx->cfg.sigma * ne);
    for (int i = 0; i < ctx->n1; ++i) T.s[i] = (float)(0.5 * (ctx->eta[i] + 1.0));
    T.start = ctx->start;
    T.rec = (const float4*)ctx->fac;
    T.field = field;
    T.counters = ctx->counters;
    const double sc = 8.0 * (double)ne * ne * ne;
    T.scale_out = (float)(sc / 4096.0);  // operands scaled by 2^8 (YZ) and 2^4 (A)
    const int td = pc_phase_begin(ctx, PC_PH_DEPOSIT);
    int nb = 0;
    e = cudaMemsetAsync(ctx->counters + CNT_ELEM, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = pc_tc_deposit_launch(T, st, &nb);
    ctx->launches += 1;
    pc_phase_end(ctx, td);
    if (e != cudaSuccess) goto fail;
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
fail:
  snprintf(ctx->err, sizeof(ctx->err), "pc_project_f32: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}

pc_status pc_collide_replay_f32_impl(pc_ctx* ctx, const pc_particles_f32* in, pc_particles_f32* out,
                                     const int32_t* partner, double dt) {
  const int64_t n = in->n;
  if (n == 0) return PC_OK;
  ReplayF32 R;
  R.n = n;
  R.nc = ctx->nc;
  R.dt = dt;
  R.e = ctx->cfg.restitution;
  R.cell = in->cell;
  R.o = in->o;
  R.v = in->v;
  R.r = in->r;
  R.m = in->m;
  R.q = in->q;
  R.id = in->id;
  R.partner = partner;
  R.cell_out = out->cell;
  R.o_out = out->o;
  R.v_out = out->v;
  R.r_out = (out->r && out->r != in->r) ? out->r : nullptr;
  R.m_out = (out->m && out->m != in->m) ? out->m : nullptr;
  R.id_out = (out->id && in->id && out->id != in->id) ? out->id : nullptr;
  R.q_out = (out->q && in->q && out->q != in->q) ? out->q : nullptr;
  R.counters = ctx->counters;
  k_replay_f32<<<pc_blocks(n, 256), 256, 0, ctx->stream>>>(R);
  ctx->launches += 1;
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_collide_replay_f32: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}

pc_status pc_collide_adjoint_f32_impl(pc_ctx* ctx, const pc_particles_f32* in, const int32_t* partner, double dt,
                                      const float* gx_out, const float* gv_out, float* gx_in, float* gv_in) {
  const int64_t n = in->n;
  if (n == 0) return PC_OK;
  AdjF32 A;
  A.n = n;
  A.nc = ctx->nc;
  A.dt = dt;
  A.e = ctx->cfg.restitution;
  A.cell = in->cell;
  A.o = in->o;
  A.v = in->v;
  A.r = in->r;
  A.m = in->m;
  A.partner = partner;
  A.gxo = gx_out;
  A.gvo = gv_out;
  A.gxi = gx_in;
  A.gvi = gv_in;
  A.counters = ctx->counters;
  k_collide_adjoint_f32<<<pc_blocks(n, 256), 256, 0, ctx->stream>>>(A);
  ctx->launches += 1;
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_collide_adjoint_f32: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}

pc_status pc_project_adjoint_f32_impl(pc_ctx* ctx, const pc_particles_f32* p, const float* G, float* gq,
                                      float* gx) {
  const int64_t n = p->n;
  if (n == 0) return PC_OK;
  const int ne = ctx->cfg.ne;
  const double rnn = (double)ne / (double)ctx->nc;
  ProjAdjF32 A;
  memset(&A, 0, sizeof(A));
  A.n = n;
  A.nc = ctx->nc;
  A.ne = ne;
  A.n1 = ctx->n1;
  A.rho = ctx->rho;
  A.win = ctx->win;
  A.rnn = {(float)rnn, (float)(rnn - (double)(float)rnn)};
  A.h = ctx->h;
  A.rc = ctx->cfg.cutoff_sigmas * ctx->cfg.sigma;
  A.rce = (float)(A.rc * ne);
  A.c2l = (float)(ctx->h * ctx->h / (2.0 * ctx->cfg.sigma * ctx->cfg.sigma) * 1.4426950408889634);
  const double s2h = 2.0 / ctx->h;
  A.scale = (float)(s2h * s2h * s2h);
  A.hs2 = (float)(ctx->h / (ctx->cfg.sigma * ctx->cfg.sigma));
  for (int w = 0; w < ctx->win; ++w)
    A.s[w] = (float)((double)(w / ctx->n1 - ctx->rho) + 0.5 * (ctx->eta[w % ctx->n1] + 1.0));
  for (int i = 0; i < ctx->n1; ++i) {
    A.wq[i] = (float)ctx->w[i];
    A.eta[i] = ctx->eta[i];
  }
  A.cell = p->cell;
  A.o = p->o;
  A.q = p->q;
  A.G = G;
  A.gq = gq;
  A.gx = gx;
  k_project_adjoint_f32<<<(unsigned)((n + 3) / 4), 128, 0, ctx->stream>>>(A);
  ctx->launches += 1;
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_project_adjoint_f32: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}
