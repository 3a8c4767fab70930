// Projection of particle sources onto the Legendre-Gauss nodes of the mesh
// (arXiv 2501.05340, Sec. 2.3 source terms, Sec. 4.2 deposition) with a Gaussian
// shape function and a box cutoff, which makes the kernel a product of 1-D
// factors: K(X - x) = kx(X_x - x_x) ky(..) kz(..), and the discrete normalisation
// Z_p = sum_g W_g K = (h/2)^3 Zx Zy Zz with Za = sum over the axis' 1-D nodes of
// w_i k_a. Hence field[g][c] = (2/h)^3 sum_p q_c (kx/Zx)(ky/Zy)(kz/Zz).
//
// Pipeline: element key + counting sort of particles by element (bin.cu), then
//   factors  per particle and axis: the normalised 1-D factors on the nodes of the
//            2 rho + 1 elements around its own element (rho = ceil(cutoff ne)),
//            in double-float; for N + 1 <= 8 written as one record per particle
//            with its per-axis reach bits and the largest factor and sources,
//   deposit  N + 1 <= 8: the per-element contraction on the tensor cores by exact
//            fixed-point digits (fx_deposit.cu); above: one CTA per element, every
//            warp takes particles of the neighbouring elements in turn and adds
//            q_c kx ky kz onto the nodes inside the particle's support box, in a
//            private shared-memory accumulator; the warps' accumulators are summed
//            in a fixed order at the end.
// No atomics: the result is deterministic for a given particle order, and the
// order is canonical (by element, then id).
#include <math.h>

#include <string.h>

#include <type_traits>

#include "df32.cuh"
#include "pc_internal.cuh"

namespace {

__device__ __forceinline__ double minimg(double d) {
  if (d > 0.5) return d - 1.0;
  if (d < -0.5) return d + 1.0;
  return d;
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

__global__ void k_elem_keys(int64_t n, const double* __restrict__ x, int ne, int32_t* __restrict__ key,
                            int32_t* __restrict__ slot, int32_t* __restrict__ cnt,
                            unsigned long long* __restrict__ counters) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x0 = x[i], x1 = x[n + i], x2 = x[2 * n + i];
  if (!((x0 >= 0.0 && x0 < 1.0) && (x1 >= 0.0 && x1 < 1.0) && (x2 >= 0.0 && x2 < 1.0)))
    atomicMax(&counters[CNT_STATUS], (unsigned long long)PC_EINVAL);
  const int k = (cell_of(x2, ne) * ne + cell_of(x1, ne)) * ne + cell_of(x0, ne);
  key[i] = k;
  slot[i] = atomicAdd(&cnt[k], 1);
}

constexpr int kMaxWin = 64;  // (2 rho + 1) n1 <= 64 (checked by pc_init)

struct FactorArgs {
  int64_t n;
  int ne, n1, rho, win;
  double h, rc;
  float rce;           // cutoff radius in element units (rc ne), float
  f2 c2;               // h^2 / (2 sigma^2): exponent factor for distances in element units
  f2 scale;            // (2/h)^3
  f2 sw[kMaxWin];      // window node offsets o + (eta_i + 1)/2 (element units), o = w/n1 - rho
  f2 wq[kMaxWin];      // Gauss weight of window node w (node w % n1)
  int wblk[kMaxWin];   // window element of node w (w / n1)
  double eta[16];      // Gauss nodes (for the exact FP64 cutoff decision)
  DfExpTable tab;
  const int32_t* perm;
  const double* x;
  const double* q;
  float2* fac;  // [3][win][n] normalised 1-D factors k_a / Z_a (df32)
  float2* sq;   // [4][n] sources times (2/h)^3 (df32)
  // record layout (tensor-core deposit, k_proj_records):
  // rec[k][rs] = the 3 win factors (axis-major), then the 4 sources; reach[k] bit
  // 8 a + w set when axis a has a non-zero factor in window element w; fxmax[0] the
  // largest factor and fxmax[1 + c] the largest |source c| (bits of non-negative
  // floats, atomically maximised)
  float2* rec;
  int rs;
  int32_t* reach;
  unsigned* fxmax;
};

// fac[a][w][k] = k_a(X_w - x_a) / Z_a over the window nodes w of the particle's
// own element and its rho neighbours on each side, k_a(d) = exp(-d^2/(2 sigma^2))
// for |d| <= rc (0 beyond), Z_a = sum_w w_i k_a. Distances are taken in element
// units relative to the own element (one FP64 subtraction per particle and axis),
// then everything runs in df32. A node whose df32 distance is within 1e-5
// relative of the cutoff is re-decided with the FP64 expression of the plain
// definition, so both sides include exactly the same nodes.
// Unnormalised factor k_a of window node w for a particle at element-relative
// position t (df32) in element ea of its axis, coordinate xa (for the FP64
// re-decision near the cutoff).
__device__ __forceinline__ f2 window_factor(const FactorArgs& F, f2 t, int ea, double xa, int w, const float* th,
                                            const float* tl) {
  const f2 dl = df_add(F.sw[w], df_neg(t));
  const float ad = fabsf(dl.h);
  bool inside;
  if (fabsf(ad - F.rce) > 1e-5f * F.rce) {
    inside = ad < F.rce;
  } else {
    const int i = w % F.n1;
    const int o = F.wblk[w] - F.rho;
    const int ge = wrapi(ea + o, F.ne);
    const double X = ((double)ge + 0.5 * (F.eta[i] + 1.0)) * F.h;
    inside = fabs(minimg(X - xa)) <= F.rc;
  }
  f2 f = {0.0f, 0.0f};
  if (inside) {
    f2 d2 = two_prod(dl.h, dl.h);
    d2.l = fmaf(2.0f * dl.h, dl.l, d2.l);
    d2 = fast_two_sum(d2.h, d2.l);
    f = df_exp_neg(df_neg(df_mul(d2, F.c2)), F.tab, th, tl);
  }
  return f;
}

// Record layout for the tensor-core deposit, WIN = (2 rho + 1) n1 window nodes per
// axis: one thread per particle, each axis' window held in registers, normalised
// and written once in 16-byte pairs; reach bits and the maxima of the digit scales.
constexpr int kRecThreads = 128;
template <int WIN>
__global__ void __launch_bounds__(kRecThreads, 4) k_proj_records(FactorArgs F) {
  __shared__ float th[64], tl[64];
  if (threadIdx.x < 64) {
    th[threadIdx.x] = F.tab.th[threadIdx.x];
    tl[threadIdx.x] = F.tab.tl[threadIdx.x];
  }
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = F.n;
  float fmax = 0.0f, qmax[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (k < n) {
    const int64_t p = F.perm[k];
    float2* rk = F.rec + k * F.rs;
    int reach = 0;
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
      const double xa = F.x[a * n + p];
      const int ea = cell_of(xa, F.ne);
      const f2 t = df_from_double(xa * (double)F.ne - (double)ea);
      f2 f[WIN];
      f2 Z = {0.0f, 0.0f};
#pragma unroll
      for (int w = 0; w < WIN; ++w) {
        f[w] = window_factor(F, t, ea, xa, w, th, tl);
        if (f[w].h != 0.0f) Z = df_add(Z, df_mul(f[w], F.wq[w]));
      }
      const f2 rz = df_recip(Z);
#pragma unroll
      for (int w = 0; w < WIN; ++w) {
        if (f[w].h != 0.0f) {
          f[w] = df_mul(f[w], rz);
          fmax = fmaxf(fmax, fabsf(f[w].h));
          reach |= 1 << (8 * a + F.wblk[w]);
        }
      }
      float2* dst = rk + a * WIN;
      if ((WIN & 1) == 0) {
#pragma unroll
        for (int w = 0; w < WIN; w += 2)
          *reinterpret_cast<float4*>(dst + w) = make_float4(f[w].h, f[w].l, f[w + 1].h, f[w + 1].l);
      } else {
#pragma unroll
        for (int w = 0; w < WIN; ++w) dst[w] = make_float2(f[w].h, f[w].l);
      }
    }
    f2 qs[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      qs[c] = df_mul(df_from_double(F.q[c * n + p]), F.scale);
      qmax[c] = fabsf(qs[c].h);
    }
    float2* dq = rk + 3 * WIN;
    if ((WIN & 1) == 0) {
      *reinterpret_cast<float4*>(dq) = make_float4(qs[0].h, qs[0].l, qs[1].h, qs[1].l);
      *reinterpret_cast<float4*>(dq + 2) = make_float4(qs[2].h, qs[2].l, qs[3].h, qs[3].l);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) dq[c] = make_float2(qs[c].h, qs[c].l);
    }
    F.reach[k] = reach;
  }
  // maxima of the float bits over the block, then one atomic per block and counter,
  // skipped when the counter already holds as much (a stale read only costs the
  // atomic): atomics of every warp on the same five words would serialise in the L2
  __shared__ unsigned red[5][kRecThreads / 32];
  const int wid = threadIdx.x >> 5;
  unsigned v = __reduce_max_sync(0xffffffffu, __float_as_uint(fmax));
  if ((threadIdx.x & 31) == 0) red[0][wid] = v;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    v = __reduce_max_sync(0xffffffffu, __float_as_uint(qmax[c]));
    if ((threadIdx.x & 31) == 0) red[1 + c][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    unsigned m = red[threadIdx.x][0];
#pragma unroll
    for (int i = 1; i < kRecThreads / 32; ++i) m = max(m, red[threadIdx.x][i]);
    if (m > *(volatile unsigned*)&F.fxmax[threadIdx.x]) atomicMax(&F.fxmax[threadIdx.x], m);
  }
}

cudaError_t launch_records(int win, const FactorArgs& F, cudaStream_t st) {
  const int nb = pc_blocks(F.n, kRecThreads);
  switch (win) {
#define PC_REC_CASE(W) \
  case W:              \
    k_proj_records<W><<<nb, kRecThreads, 0, st>>>(F); \
    return cudaGetLastError();
    PC_REC_CASE(3) PC_REC_CASE(5) PC_REC_CASE(6) PC_REC_CASE(9) PC_REC_CASE(10) PC_REC_CASE(12) PC_REC_CASE(15)
    PC_REC_CASE(18) PC_REC_CASE(20) PC_REC_CASE(21) PC_REC_CASE(24) PC_REC_CASE(25) PC_REC_CASE(30) PC_REC_CASE(35)
    PC_REC_CASE(40)
#undef PC_REC_CASE
    default: return cudaErrorInvalidValue;
  }
}

__global__ void __launch_bounds__(128) k_proj_factors(FactorArgs F) {
  __shared__ float th[64], tl[64];
  if (threadIdx.x < 64) {
    th[threadIdx.x] = F.tab.th[threadIdx.x];
    tl[threadIdx.x] = F.tab.tl[threadIdx.x];
  }
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = F.n;
  if (k >= n) return;
  const int64_t p = F.perm[k];
  for (int a = 0; a < 3; ++a) {
    const double xa = F.x[a * n + p];
    const int ea = cell_of(xa, F.ne);
    const f2 t = df_from_double(xa * (double)F.ne - (double)ea);
    f2 Z = {0.0f, 0.0f};
    for (int w = 0; w < F.win; ++w) {
      const f2 f = window_factor(F, t, ea, xa, w, th, tl);
      if (f.h != 0.0f) Z = df_add(Z, df_mul(f, F.wq[w]));
      F.fac[((int64_t)a * F.win + w) * n + k] = make_float2(f.h, f.l);
    }
    const f2 rz = df_recip(Z);
    for (int w = 0; w < F.win; ++w) {
      float2* slot = &F.fac[((int64_t)a * F.win + w) * n + k];
      const float2 v = *slot;
      if (v.x != 0.0f) {
        const f2 r = df_mul({v.x, v.y}, rz);
        *slot = make_float2(r.h, r.l);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const f2 qs = df_mul(df_from_double(F.q[c * n + p]), F.scale);
    F.sq[c * n + k] = make_float2(qs.h, qs.l);
  }
}

struct DepositArgs {
  int64_t n;
  int ne, n1, rho, win, nwarps, batch;
  unsigned Mraw, Mper, Mn1;  // recip_of(3 n1 + 4), recip_of(4 n1 + n1^2), recip_of(n1)
  const int32_t* start;
  const float2* fac;
  const float2* sq;
  double* field;
};

// floor(t / d) for t < 2^32 / d via a 32-bit reciprocal M = ceil(2^32 / d); the
// reciprocal of d = 1 does not fit in 32 bits and is encoded as 0.
__device__ __forceinline__ unsigned div_by(unsigned t, unsigned M) { return M ? __umulhi(t, M) : t; }
__host__ __device__ __forceinline__ unsigned recip_of(unsigned d) {
  return d <= 1 ? 0u : (unsigned)((0x100000000ull + d - 1) / d);
}

// One CTA per element. The particles of the (2 rho + 1)^3 neighbouring elements are
// taken in batches of BS; batch b goes to warp b mod NW. Staging is spread over the
// warp's lanes: (S0) per particle its index and factor-window offsets, (S1) the
// factor slices on this element's nodes and the sources, (S2) the support box,
// (S3) the df32 products A[c][i] = q_c kx_i and YZ[row] = ky_j kz_k. (S4) all lanes
// sweep each staged particle's support box, adding A YZ onto a warp-private df32
// accumulator in shared memory (TwoSum on the high part, errors summed in the low
// part). The warps' accumulators are added in a fixed order at the end, so the
// result does not depend on scheduling.
__global__ void k_proj_deposit(DepositArgs G) {
  extern __shared__ float2 sm2[];
  const int n1 = G.n1, nodes = n1 * n1 * n1, NW = G.nwarps, BS = G.batch;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_p = 4 * n1 + n1 * n1;  // A and YZ per particle
  const int raw_p = 3 * n1 + 4;        // factor slices + sources per particle
  float2* acc = sm2;                                                  // [NW][4][nodes]
  float2* stage = acc + (size_t)NW * 4 * nodes;                       // [NW][BS][per_p]
  float2* raw = stage + (size_t)NW * BS * per_p;                      // [NW][BS][raw_p]
  int* meta = (int*)(raw + (size_t)NW * BS * raw_p);                  // [NW][BS][4]: j, wo0, wo1, wo2
  int* bx = meta + NW * BS * 4;                                       // [NW][BS]: packed box (or -1)
  int* pre = bx + NW * BS;                                            // [126] prefix of range sizes
  int* rbeg = pre + 126;                                              // [125] range starts
  unsigned* rtab = (unsigned*)(rbeg + 125);                           // [33] recip_of(d), d = 0..32
  float2* my = acc + (size_t)warp * 4 * nodes;
  float2* st = stage + (size_t)warp * BS * per_p;
  float2* rw = raw + (size_t)warp * BS * raw_p;
  int* mt = meta + warp * BS * 4;
  int* bw = bx + warp * BS;
  for (int a = threadIdx.x; a < NW * 4 * nodes; a += blockDim.x) acc[a] = make_float2(0.0f, 0.0f);
  if (threadIdx.x < 33) rtab[threadIdx.x] = recip_of(threadIdx.x);
  const int64_t n = G.n;
  const int ne = G.ne, rho = G.rho, span = 2 * rho + 1, nrange = span * span * span;
  const int e = blockIdx.x;
  const int ex = e % ne, ey = (e / ne) % ne, ez = e / (ne * ne);
  if (threadIdx.x == 0) {
    int s = 0;
    for (int r = 0; r < nrange; ++r) {
      const int dx = r % span - rho, dy = (r / span) % span - rho, dz = r / (span * span) - rho;
      const int nb = (wrapi(ez + dz, ne) * ne + wrapi(ey + dy, ne)) * ne + wrapi(ex + dx, ne);
      const int b0 = G.start[nb], b1 = G.start[nb + 1];
      pre[r] = s;
      rbeg[r] = b0;
      s += b1 - b0;
    }
    pre[nrange] = s;
  }
  __syncthreads();
  const int total = pre[nrange];
  const int nbatch = (total + BS - 1) / BS;
  const unsigned Mraw = G.Mraw, Mper = G.Mper, Mn1 = G.Mn1;
  for (int b = warp; b < nbatch; b += NW) {
    // S0: particle index and window offsets
    if (lane < BS) {
      const int idx = b * BS + lane;
      int j = -1, w0 = 0, w1 = 0, w2 = 0;
      if (idx < total) {
        int r = 0;
        while (pre[r + 1] <= idx) ++r;
        j = rbeg[r] + (idx - pre[r]);
        w0 = (rho - (r % span - rho)) * n1;
        w1 = (rho - ((r / span) % span - rho)) * n1;
        w2 = (rho - (r / (span * span) - rho)) * n1;
      }
      mt[4 * lane] = j;
      mt[4 * lane + 1] = w0;
      mt[4 * lane + 2] = w1;
      mt[4 * lane + 3] = w2;
    }
    __syncwarp();
    // S1: factor slices and sources
    for (int t = lane; t < BS * raw_p; t += 32) {
      const int p = (int)div_by((unsigned)t, Mraw);
      const int r = t - p * raw_p;
      const int j = mt[4 * p];
      float2 v = make_float2(0.0f, 0.0f);
      if (j >= 0) {
        if (r < 3 * n1) {
          const int a = (int)div_by((unsigned)r, Mn1);
          const int i = r - a * n1;
          v = G.fac[((int64_t)a * G.win + mt[4 * p + 1 + a] + i) * n + j];
        } else {
          v = G.sq[(int64_t)(r - 3 * n1) * n + j];
        }
      }
      rw[t] = v;
    }
    __syncwarp();
    // S2: support box of each particle on this element
    if (lane < BS) {
      const float2* f = rw + lane * raw_p;
      int lo[3], cnt[3];
      for (int a = 0; a < 3; ++a) {
        int l = -1, h = -2;
        for (int i = 0; i < n1; ++i)
          if (f[a * n1 + i].x != 0.0f) {
            if (l < 0) l = i;
            h = i;
          }
        lo[a] = l < 0 ? 0 : l;
        cnt[a] = h >= l ? h - l + 1 : 0;
      }
      bw[lane] = (mt[4 * lane] >= 0 && cnt[0] && cnt[1] && cnt[2])
                     ? (lo[0] | (cnt[0] << 5) | (lo[1] << 10) | (cnt[1] << 15) | (lo[2] << 20) | (cnt[2] << 25))
                     : -1;
    }
    __syncwarp();
    // S3: products
    for (int t = lane; t < BS * per_p; t += 32) {
      const int p = (int)div_by((unsigned)t, Mper);
      const int box = bw[p];
      if (box < 0) continue;
      const int r = t - p * per_p;
      const float2* f = rw + p * raw_p;
      const int lx = box & 31, cx = (box >> 5) & 31, ly = (box >> 10) & 31, cy = (box >> 15) & 31;
      const int lz = (box >> 20) & 31, cz = (box >> 25) & 31;
      if (r < 4 * n1) {
        const int c = (int)div_by((unsigned)r, Mn1);
        const int ii = r - c * n1;
        if (ii < cx) {
          const float2 fx = f[lx + ii], qv = f[3 * n1 + c];
          const f2 v = df_mul({qv.x, qv.y}, {fx.x, fx.y});
          st[p * per_p + r] = make_float2(v.h, v.l);
        }
      } else {
        const int row = r - 4 * n1;
        if (row < cy * cz) {
          const int kk = (int)div_by((unsigned)row, rtab[cy]);
          const int jj = row - kk * cy;
          const float2 fy = f[n1 + ly + jj], fz = f[2 * n1 + lz + kk];
          const f2 v = df_mul({fy.x, fy.y}, {fz.x, fz.y});
          st[p * per_p + r] = make_float2(v.h, v.l);
        }
      }
    }
    __syncwarp();
    // S4: sweep the support box of each staged particle
    for (int q = 0; q < BS; ++q) {
      const int box = bw[q];
      if (box < 0) continue;
      const int lx = box & 31, cx = (box >> 5) & 31, ly = (box >> 10) & 31, cy = (box >> 15) & 31;
      const int lz = (box >> 20) & 31, cz = (box >> 25) & 31;
      const int nbox = cx * cy * cz;
      const unsigned Mx = rtab[cx], My = rtab[cy];
      const float2* sp = st + (size_t)q * per_p;
      for (int u = lane; u < nbox; u += 32) {
        const int row = (int)div_by((unsigned)u, Mx);
        const int ii = u - row * cx;
        const int kk = (int)div_by((unsigned)row, My);
        const int jj = row - kk * cy;
        const int g = ((lz + kk) * n1 + ly + jj) * n1 + lx + ii;
        const float2 yz = sp[4 * n1 + row];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float2 a = sp[c * n1 + ii];
          const float pp = a.x * yz.x;
          float pe = fmaf(a.x, yz.x, -pp);
          pe = fmaf(a.x, yz.y, pe);
          pe = fmaf(a.y, yz.x, pe);
          float2 S = my[c * nodes + g];
          const f2 s = two_sum(S.x, pp);
          S.x = s.h;
          S.y += s.l + pe;
          my[c * nodes + g] = S;
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
  double* out = G.field + (int64_t)e * 4 * nodes;
  for (int a = threadIdx.x; a < 4 * nodes; a += blockDim.x) {
    f2 s = {0.0f, 0.0f};
    for (int w = 0; w < NW; ++w) {
      const float2 v = acc[(size_t)w * 4 * nodes + a];
      s = df_add(s, {v.x, v.y});
    }
    out[a] = df_to_double(s);
  }
}

}  // namespace

static void deposit_shape(int n1, int* nwarps, int* batch, size_t* smem) {
  const size_t nodes = (size_t)n1 * n1 * n1;
  const size_t per_p = 4 * (size_t)n1 + (size_t)n1 * n1, raw_p = 3 * (size_t)n1 + 4;
  const size_t budget = 200 * 1024;
  const size_t fixed = (126 + 125 + 33) * sizeof(int) + 64;
  static const int kWarps[] = {16, 12, 8, 6, 4, 2, 1};
  for (int nw : kWarps)
    for (int bs = 32; bs >= 8; bs /= 2) {
      const size_t need = nw * (4 * nodes + bs * (per_p + raw_p)) * sizeof(float2) + nw * bs * 5 * sizeof(int) + fixed;
      if (need <= budget) {
        *nwarps = nw;
        *batch = bs;
        *smem = need;
        return;
      }
    }
  *nwarps = 1;
  *batch = 8;
  *smem = (4 * nodes + 8 * (per_p + raw_p)) * sizeof(float2) + 8 * 5 * sizeof(int) + fixed;
}

cudaError_t pc_elem_bin(pc_ctx* ctx, int64_t n, const double* x, const int32_t* id) {
  cudaStream_t st = ctx->stream;
  const int ne = ctx->cfg.ne;
  const int64_t nel = (int64_t)ne * ne * ne;
  PC_CUDA_TRY(cudaMemsetAsync(ctx->cnt, 0, sizeof(int32_t) * (size_t)nel, st));
  const int tb = pc_phase_begin(ctx, PC_PH_PBIN);
  if (n > 0) {
    k_elem_keys<<<pc_blocks(n, 256), 256, 0, st>>>(n, x, ne, ctx->key, ctx->slot, ctx->cnt, ctx->counters);
    ctx->launches += 1;
  }
  const cudaError_t e = pc_bin_finish(n, nel, ctx->key, ctx->slot, id, ctx->cnt, ctx->start, ctx->blocksums,
                                      ctx->perm, st, &ctx->launches);
  pc_phase_end(ctx, tb);
  return e;
}

pc_status pc_project_impl(pc_ctx* ctx, const pc_particles* p, double* field) {
  const int64_t n = p->n;
  cudaStream_t st = ctx->stream;
  const int ne = ctx->cfg.ne;
  const int64_t nel = (int64_t)ne * ne * ne;
  cudaError_t e = pc_elem_bin(ctx, n, p->x, p->id);
  if (e != cudaSuccess) goto fail;
  if (n > 0) {
    FactorArgs F;
    memset(&F, 0, sizeof(F));
    F.n = n;
    F.ne = ne;
    F.n1 = ctx->n1;
    F.rho = ctx->rho;
    F.win = ctx->win;
    F.h = ctx->h;
    F.rc = ctx->cfg.cutoff_sigmas * ctx->cfg.sigma;
    F.rce = (float)(F.rc * ne);
    const double c2 = ctx->h * ctx->h / (2.0 * ctx->cfg.sigma * ctx->cfg.sigma);
    F.c2 = {(float)c2, (float)(c2 - (double)(float)c2)};
    const double sc = 8.0 * (double)ne * ne * ne;
    F.scale = {(float)sc, (float)(sc - (double)(float)sc)};
    for (int w = 0; w < ctx->win; ++w) {
      const double v = (double)(w / ctx->n1 - ctx->rho) + 0.5 * (ctx->eta[w % ctx->n1] + 1.0);
      F.sw[w] = {(float)v, (float)(v - (double)(float)v)};
      const double wq = ctx->w[w % ctx->n1];
      F.wq[w] = {(float)wq, (float)(wq - (double)(float)wq)};
      F.wblk[w] = w / ctx->n1;
    }
    for (int i = 0; i < ctx->n1; ++i) F.eta[i] = ctx->eta[i];
    F.tab = ctx->exp_tab;
    F.perm = ctx->perm;
    F.x = p->x;
    F.q = p->q;
    F.fac = ctx->fac;
    F.sq = ctx->sq;
    if (ctx->n1 <= 8) {
      F.rec = ctx->fac;
      F.rs = ctx->rs;
      F.reach = ctx->reach;
      F.fxmax = ctx->fxmax;
      e = cudaMemsetAsync(ctx->fxmax, 0, sizeof(unsigned) * 8, st);
      if (e != cudaSuccess) goto fail;
    }
    const int tf = pc_phase_begin(ctx, PC_PH_FACTORS);
    if (ctx->n1 <= 8) {
      e = launch_records(ctx->win, F, st);
      if (e != cudaSuccess) goto fail;
    } else {
      k_proj_factors<<<pc_blocks(n, 128), 128, 0, st>>>(F);
    }
    ctx->launches += 1;
    pc_phase_end(ctx, tf);
  }
  {
    DepositArgs G;
    G.n = n;
    G.ne = ne;
    G.n1 = ctx->n1;
    G.rho = ctx->rho;
    G.win = ctx->win;
    size_t smem = 0;
    deposit_shape(ctx->n1, &G.nwarps, &G.batch, &smem);
    G.Mraw = recip_of(3 * ctx->n1 + 4);
    G.Mper = recip_of(4 * ctx->n1 + ctx->n1 * ctx->n1);
    G.Mn1 = recip_of(ctx->n1);
    G.start = ctx->start;
    G.fac = ctx->fac;
    G.sq = ctx->sq;
    G.field = field;
    if (ctx->n1 <= 8) {
      if (n == 0) {  // no records: every element's deposit is zero
        e = cudaMemsetAsync(ctx->fxmax, 0, sizeof(unsigned) * 8, st);
        if (e != cudaSuccess) goto fail;
      }
      const int td = pc_phase_begin(ctx, PC_PH_DEPOSIT);
      e = pc_fx_deposit_launch(ctx->n1, ne, ctx->rho, ctx->win, ctx->rs, ctx->start, ctx->fac, ctx->reach, ctx->fxmax,
                               field, ctx->counters, st);
      ctx->launches += 1;
      pc_phase_end(ctx, td);
      if (e != cudaSuccess) goto fail;
    } else {
      e = cudaFuncSetAttribute(k_proj_deposit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) goto fail;
      const int td = pc_phase_begin(ctx, PC_PH_DEPOSIT);
      k_proj_deposit<<<(unsigned)nel, 32 * G.nwarps, smem, st>>>(G);
      ctx->launches += 1;
      pc_phase_end(ctx, td);
    }
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
fail:
  snprintf(ctx->err, sizeof(ctx->err), "pc_project: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}
