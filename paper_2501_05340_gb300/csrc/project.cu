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
//   gather   one CTA per element: every warp takes particles of the neighbouring
//            elements in turn and adds q_c kx ky kz onto the nodes inside the
//            particle's support box, in a private shared-memory accumulator; the
//            warps' accumulators are summed in a fixed order at the end.
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
  f2 wq[16];           // Gauss weights
  double eta[16];      // Gauss nodes (for the exact FP64 cutoff decision)
  DfExpTable tab;
  const int32_t* perm;
  const double* x;
  const double* q;
  float2* fac;  // [3][win][n] normalised 1-D factors k_a / Z_a (df32)
  float2* sq;   // [4][n] sources times (2/h)^3 (df32)
};

// fac[a][w][k] = k_a(X_w - x_a) / Z_a over the window nodes w of the particle's
// own element and its rho neighbours on each side, k_a(d) = exp(-d^2/(2 sigma^2))
// for |d| <= rc (0 beyond), Z_a = sum_w w_i k_a. Distances are taken in element
// units relative to the own element (one FP64 subtraction per particle and axis),
// then everything runs in df32. A node whose df32 distance is within 1e-5
// relative of the cutoff is re-decided with the FP64 expression of the plain
// definition, so both sides include exactly the same nodes.
__global__ void __launch_bounds__(128) k_proj_factors(FactorArgs F) {
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
      const int i = w % F.n1;
      const f2 dl = df_add(F.sw[w], df_neg(t));
      const float ad = fabsf(dl.h);
      bool inside;
      if (fabsf(ad - F.rce) > 1e-5f * F.rce) {
        inside = ad < F.rce;
      } else {
        const int o = w / F.n1 - F.rho;
        const int ge = wrapi(ea + o, F.ne);
        const double X = ((double)ge + 0.5 * (F.eta[i] + 1.0)) * F.h;
        inside = fabs(minimg(X - xa)) <= F.rc;
      }
      f2 f = {0.0f, 0.0f};
      if (inside) {
        f2 d2 = two_prod(dl.h, dl.h);
        d2.l = fmaf(2.0f * dl.h, dl.l, d2.l);
        d2 = fast_two_sum(d2.h, d2.l);
        f = df_exp_neg(df_neg(df_mul(d2, F.c2)), F.tab);
        Z = df_add(Z, df_mul(f, F.wq[i]));
      }
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

// ---- blocked deposit, n1 <= 8 -------------------------------------------------
// An element's deposit is the contraction D[jk][ci] = sum_p YZ_p[jk] A_p[ci] with
// YZ = ky_j kz_k and A = q_c kx_i (df32), jk = k n1 + j, ci = c n1 + i. One CTA per
// element and one warp per 2 x 2 block of (j, k) node lines; lane (b, g) of a warp
// owns (j, k) = (2 wj + (b & 1), 2 wk + (b >> 1)), b = lane >> 3, and the TC columns
// ci = g TC .. g TC + TC - 1, g = lane & 7, as df32 accumulators in registers. A
// warp runs only over the staged particles whose y and z support meets its lines:
// outside the support the factors are exact zeros, so the skipped terms change no
// sum. Candidates come in batches of 32 (in a fixed permuted order that spreads
// each batch over the neighbourhood), staged lane-per-candidate into a double
// buffer; every sum runs in that order, so the result is deterministic.
template <int N1>
struct BlkShape {
  static constexpr int NB = (N1 + 1) / 2;          // blocks per side
  static constexpr int NW = NB * NB;               // warps per CTA
  static constexpr int TC = (4 * N1 + 7) / 8;      // columns per lane
  static constexpr int TCP = TC == 3 ? 4 : TC;     // padded column group
  static constexpr int YZP = (N1 * N1 + 1) & ~1;   // YZ entries, padded to 16 bytes
  // staged df32 values per particle: YZ, then A as [TCP / 2][8 groups][2] (groups of
  // one column when TCP = 1); the row pitch in 16-byte units is odd, so that the
  // stager's per-lane row stores do not collide in the banks
  static constexpr int PER0 = YZP + 8 * TCP;
  static constexpr int PER = (PER0 / 2) % 2 == 1 ? PER0 : PER0 + 2;
  static constexpr int MINB = NW == 1 ? 16 : (NW == 4 ? 8 : (NW == 9 ? 4 : 2));
  static constexpr size_t SMEM = (size_t)(2 * 32 * PER + PER) * sizeof(float2) + (size_t)(2 * 32 + 376) * sizeof(int);
};

struct BlkArgs {
  int64_t n;
  int ne, rho, win;
  const int32_t* start;
  const float2* fac;
  const float2* sq;
  double* field;
};

// acc += a b for df32 a, b: product with its FMA error terms, TwoSum on the high
// parts, all errors gathered in the low part.
__device__ __forceinline__ void df_fma_acc(f2& acc, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float s = acc.h + p;
  const float bb = s - acc.h;
  const float err = (acc.h - (s - bb)) + (p - bb);
  acc.h = s;
  acc.l = acc.l + (err + e);
}

// Two accumulators at once on the packed FP32x2 pipe instructions: (H, L) += (ah, al) b
// with H, L, ah, al pairs of high and low parts and b one df32 value; the same
// operations as df_fma_acc, lane by lane.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void df_fma_acc2(float2& H, float2& L, float2 ah, float2 al, float2 b) {
  const float2 bh = make_float2(b.x, b.x), bl = make_float2(b.y, b.y);
  const float2 p = __fmul2_rn(ah, bh);
  float2 e = __ffma2_rn(ah, bh, neg2(p));
  e = __ffma2_rn(ah, bl, e);
  e = __ffma2_rn(al, bh, e);
  const float2 s = __fadd2_rn(H, p);
  const float2 bb = __fadd2_rn(s, neg2(H));
  const float2 err = __fadd2_rn(__fadd2_rn(H, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(p, neg2(bb)));
  H = s;
  L = __fadd2_rn(L, __fadd2_rn(err, e));
}

__device__ __forceinline__ float2 df_mul2(float2 a, float2 b) {
  const f2 v = df_mul({a.x, a.y}, {b.x, b.y});
  return make_float2(v.h, v.l);
}

// Offset of A column (group g, slot t) in a staged row.
template <int N1>
__host__ __device__ constexpr int a_off(int g, int t) {
  using B = BlkShape<N1>;
  return B::TCP == 1 ? B::YZP + g : B::YZP + ((t >> 1) * 8 + g) * 2 + (t & 1);
}

// Column ci held at entry x of the A part of a staged row (inverse of a_off), or -1
// for padding.
template <int N1>
__host__ __device__ constexpr int a_col(int x) {
  using B = BlkShape<N1>;
  const int g = B::TCP == 1 ? x : (B::TCP == 2 ? x / 2 : (x / 2) % 8);
  const int t = B::TCP == 1 ? 0 : (B::TCP == 2 ? x % 2 : 2 * ((x / 2) / 8) + x % 2);
  const int ci = g * B::TC + t;
  return (t < B::TC && ci < 4 * N1) ? ci : -1;
}

template <int N1>
__global__ void __launch_bounds__(32 * BlkShape<N1>::NW, BlkShape<N1>::MINB) k_proj_deposit_blk(BlkArgs G) {
  using B = BlkShape<N1>;
  constexpr int NW = B::NW, TC = B::TC, TCP = B::TCP, PER = B::PER, YZP = B::YZP;
  constexpr int NODES = N1 * N1 * N1;
  extern __shared__ float4 smb4[];
  float2* stage = reinterpret_cast<float2*>(smb4);          // [2][32][PER]
  float2* zrow = stage + 2 * 32 * PER;                      // [PER] zeros: the partner of an odd last particle
  int* box = reinterpret_cast<int*>(zrow + PER);            // [2][32]: y, z support lines; -1 if not kept
  int* pre = box + 2 * 32;                                  // [126] prefix of the neighbour range sizes
  int* rbeg = pre + 126;                                    // [125]
  int* rmeta = rbeg + 125;                                  // [125]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = G.n;
  const int ne = G.ne, rho = G.rho, span = 2 * rho + 1, nrange = span * span * span, win = G.win;
  const int e = blockIdx.x;
  const int ex = e % ne, ey = (e / ne) % ne, ez = e / (ne * ne);
  for (int t = threadIdx.x; t < PER; t += blockDim.x) zrow[t] = make_float2(0.0f, 0.0f);
  if (warp == 0) {
    int tot = 0;
    for (int r0 = 0; r0 < nrange; r0 += 32) {
      const int r = r0 + lane;
      int cnt = 0;
      if (r < nrange) {
        const int dx = r % span - rho, dy = (r / span) % span - rho, dz = r / (span * span) - rho;
        const int nb = (wrapi(ez + dz, ne) * ne + wrapi(ey + dy, ne)) * ne + wrapi(ex + dx, ne);
        const int b0 = G.start[nb];
        cnt = G.start[nb + 1] - b0;
        rbeg[r] = b0;
        rmeta[r] = ((rho - dx) * N1) | (((rho - dy) * N1) << 8) | (((rho - dz) * N1) << 16);
      }
      int x = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (r < nrange) pre[r + 1] = tot + x;
      tot += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) pre[0] = 0;
  }
  __syncthreads();
  const int total = pre[nrange];
  const int nbatch = (total + 31) / 32;
  int top = 1;
  while (2 * top < nrange) top *= 2;
  // Candidates are taken in blocks of 8 whose order is a multiplicative permutation
  // blk -> blk mix mod nfull (mix coprime to nfull, near nfull / golden ratio), so that
  // a batch mixes four distant blocks of the neighbourhood and the warps' shares of a
  // batch stay even; the trailing partial block keeps its place.
  const int nfull = total >> 3;
  int mix = 1;
  if (nfull > 2) {
    mix = (int)(0.6180339887 * nfull) | 1;
    for (;; mix += 2) {
      int a = nfull, c = mix;
      while (c) {
        const int t = a % c;
        a = c;
        c = t;
      }
      if (a == 1) break;
    }
  }

  // Staging of batch b into buffer buf, lane = candidate, in three parts that go to
  // three different warps: part 0 and 1 the YZ products of the lower and upper k half,
  // part 2 the A products and the support box.
  auto cand = [&](int b, int64_t& jj, int& wm) -> bool {
    int idx = b * 32 + lane;
    jj = 0;
    wm = 0;
    if (idx >= total) return false;
    if ((idx >> 3) < nfull) idx = (int)(((int64_t)(idx >> 3) * mix) % nfull) * 8 + (idx & 7);
    int r = 0;
    for (int stp = top; stp > 0; stp >>= 1)
      if (r + stp < nrange && pre[r + stp] <= idx) r += stp;
    jj = rbeg[r] + (idx - pre[r]);
    wm = rmeta[r];
    return true;
  };
  auto stage_yz = [&](int b, int buf, auto half) {
    constexpr int H = decltype(half)::value;
    constexpr int KH = (N1 + 1) / 2;                       // k lines in the lower half
    constexpr int U0 = H == 0 ? 0 : (KH * N1) / 2;         // float4 range of this half
    constexpr int U1 = H == 0 ? (KH * N1) / 2 : YZP / 2;
    int64_t jj;
    int wm;
    const bool valid = cand(b, jj, wm);
    float4* row = reinterpret_cast<float4*>(stage + (size_t)(buf * 32 + lane) * PER);
    float2 fy[N1], fz[N1];
    const float2* py = G.fac + ((int64_t)win + ((wm >> 8) & 255)) * n + jj;
    const float2* pz = G.fac + ((int64_t)2 * win + ((wm >> 16) & 255)) * n + jj;
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      fy[i] = valid ? py[(int64_t)i * n] : make_float2(0.0f, 0.0f);
      const bool need = (2 * U0) / N1 <= i && i <= (2 * U1 - 1) / N1;
      fz[i] = (valid && need) ? pz[(int64_t)i * n] : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int u = U0; u < U1; ++u) {
      float2 v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int q = 2 * u + h;
        v[h] = q < N1 * N1 ? df_mul2(fy[q % N1], fz[q / N1]) : make_float2(0.0f, 0.0f);
      }
      row[u] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    }
  };
  auto stage_a = [&](int b, int buf) {
    int64_t jj;
    int wm;
    const bool valid = cand(b, jj, wm);
    float4* row = reinterpret_cast<float4*>(stage + (size_t)(buf * 32 + lane) * PER);
    int ylo = N1, yhi = -1, zlo = N1, zhi = -1;
    {
      const float* py = reinterpret_cast<const float*>(G.fac + ((int64_t)win + ((wm >> 8) & 255)) * n + jj);
      const float* pz = reinterpret_cast<const float*>(G.fac + ((int64_t)2 * win + ((wm >> 16) & 255)) * n + jj);
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        const float y = valid ? py[2 * (int64_t)i * n] : 0.0f;
        const float z = valid ? pz[2 * (int64_t)i * n] : 0.0f;
        if (y != 0.0f) {
          ylo = min(ylo, i);
          yhi = i;
        }
        if (z != 0.0f) {
          zlo = min(zlo, i);
          zhi = i;
        }
      }
    }
    float2 fx[N1], qv[4];
    bool xany = false;
    const float2* px = G.fac + (int64_t)(wm & 255) * n + jj;
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      fx[i] = valid ? px[(int64_t)i * n] : make_float2(0.0f, 0.0f);
      xany = xany || fx[i].x != 0.0f;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) qv[c] = valid ? G.sq[(int64_t)c * n + jj] : make_float2(0.0f, 0.0f);
#pragma unroll
    for (int u = 0; u < 4 * TCP; ++u) {
      float2 v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ci = a_col<N1>(2 * u + h);
        v[h] = ci >= 0 ? df_mul2(qv[ci / N1], fx[ci % N1]) : make_float2(0.0f, 0.0f);
      }
      // column pairs of a group as (h0, h1, l0, l1) for the packed accumulators
      row[YZP / 2 + u] = TCP == 1 ? make_float4(v[0].x, v[0].y, v[1].x, v[1].y)
                                  : make_float4(v[0].x, v[1].x, v[0].y, v[1].y);
    }
    box[buf * 32 + lane] = (yhi >= 0 && zhi >= 0 && xany) ? (ylo | (yhi << 8) | (zlo << 16) | (zhi << 24)) : -1;
  };
  // the parts of batch b go to warps 3 b, 3 b + 1, 3 b + 2 (mod NW)
  auto stage_parts = [&](int b) {
    const int buf = b & 1;
#pragma unroll
    for (int part = 0; part < 3; ++part) {
      if (warp != (3 * b + part) % NW) continue;
      if (part == 0) stage_yz(b, buf, std::integral_constant<int, 0>());
      if (part == 1) stage_yz(b, buf, std::integral_constant<int, 1>());
      if (part == 2) stage_a(b, buf);
    }
  };

  // this lane's outputs and their staged-row offsets
  const int wj = warp % B::NB, wk = warp / B::NB;
  const int bq = lane >> 3, g = lane & 7;
  const int j = 2 * wj + (bq & 1), k = 2 * wk + (bq >> 1);
  const bool jk_ok = j < N1 && k < N1;
  const int jk = jk_ok ? k * N1 + j : 0;
  const int y0 = 2 * wj, z0 = 2 * wk;
  // columns 2u, 2u + 1 of this lane in packed pairs (H, L); an odd last column in acc1
  constexpr int NP = TC / 2;
  float2 AH[NP > 0 ? NP : 1], AL[NP > 0 ? NP : 1];
#pragma unroll
  for (int u = 0; u < (NP > 0 ? NP : 1); ++u) AH[u] = AL[u] = make_float2(0.0f, 0.0f);
  f2 acc1 = {0.0f, 0.0f};
  auto gemm_batch = [&](int buf) {
    const float2* sb = stage + (size_t)buf * 32 * PER;
    const int w = box[buf * 32 + lane];
    const int ylo = w & 255, yhi = (w >> 8) & 255, zlo = (w >> 16) & 255, zhi = (w >> 24) & 255;
    const bool rel = w >= 0 && ylo <= y0 + 1 && yhi >= y0 && zlo <= z0 + 1 && zhi >= z0;
    unsigned m = __ballot_sync(0xffffffffu, rel);
    // two particles per pass; an odd last one is paired with the zero row, whose
    // terms leave the accumulators bit for bit unchanged
    while (m) {
      const float2* pr[2];
      pr[0] = sb + (__ffs(m) - 1) * PER;
      m &= m - 1;
      pr[1] = m ? sb + (__ffs(m) - 1) * PER : zrow;
      m &= m - 1;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
      const float2* pq = pr[h];
      const float2 bv = pq[jk];
      if constexpr (TCP == 1) {
        df_fma_acc(acc1, pq[YZP + g], bv);
      } else {
#pragma unroll
        for (int u = 0; u < TCP / 2; ++u) {
          const float4 v4 = *reinterpret_cast<const float4*>(pq + a_off<N1>(g, 2 * u));
          if (2 * u + 1 < TC)
            df_fma_acc2(AH[u], AL[u], make_float2(v4.x, v4.y), make_float2(v4.z, v4.w), bv);
          else if (2 * u < TC)
            df_fma_acc(acc1, make_float2(v4.x, v4.z), bv);
        }
      }
      }
    }
  };

  if (nbatch > 0) stage_parts(0);
  __syncthreads();
  for (int b = 0; b < nbatch; ++b) {
    if (b + 1 < nbatch) stage_parts(b + 1);
    gemm_batch(b & 1);
    __syncthreads();
  }
  if (jk_ok) {
    double* out = G.field + (int64_t)e * 4 * NODES;
#pragma unroll
    for (int t = 0; t < TC; ++t) {
      const int ci = g * TC + t;
      if (ci < 4 * N1) {
        const int c = ci / N1, i = ci - c * N1;
        float h, l;
        if (TCP == 1 || t >= 2 * NP) {
          h = acc1.h;
          l = acc1.l;
        } else {
          h = (t & 1) ? AH[t / 2].y : AH[t / 2].x;
          l = (t & 1) ? AL[t / 2].y : AL[t / 2].x;
        }
        out[c * NODES + jk * N1 + i] = (double)h + (double)l;
      }
    }
  }
}

template <int N1>
cudaError_t launch_blk(const BlkArgs& G, int64_t nel, cudaStream_t st) {
  using B = BlkShape<N1>;
  cudaError_t e = cudaFuncSetAttribute(k_proj_deposit_blk<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B::SMEM);
  if (e != cudaSuccess) return e;
  k_proj_deposit_blk<N1><<<(unsigned)nel, 32 * B::NW, B::SMEM, st>>>(G);
  return cudaGetLastError();
}

cudaError_t launch_blk_n1(int n1, const BlkArgs& G, int64_t nel, cudaStream_t st) {
  switch (n1) {
    case 1: return launch_blk<1>(G, nel, st);
    case 2: return launch_blk<2>(G, nel, st);
    case 3: return launch_blk<3>(G, nel, st);
    case 4: return launch_blk<4>(G, nel, st);
    case 5: return launch_blk<5>(G, nel, st);
    case 6: return launch_blk<6>(G, nel, st);
    case 7: return launch_blk<7>(G, nel, st);
    case 8: return launch_blk<8>(G, nel, st);
    default: return cudaErrorInvalidValue;
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
    }
    for (int i = 0; i < ctx->n1; ++i) {
      F.wq[i] = {(float)ctx->w[i], (float)(ctx->w[i] - (double)(float)ctx->w[i])};
      F.eta[i] = ctx->eta[i];
    }
    F.tab = ctx->exp_tab;
    F.perm = ctx->perm;
    F.x = p->x;
    F.q = p->q;
    F.fac = ctx->fac;
    F.sq = ctx->sq;
    const int tf = pc_phase_begin(ctx, PC_PH_FACTORS);
    k_proj_factors<<<pc_blocks(n, 128), 128, 0, st>>>(F);
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
      BlkArgs K;
      K.n = n;
      K.ne = ne;
      K.rho = ctx->rho;
      K.win = ctx->win;
      K.start = ctx->start;
      K.fac = ctx->fac;
      K.sq = ctx->sq;
      K.field = field;
      const int td = pc_phase_begin(ctx, PC_PH_DEPOSIT);
      e = launch_blk_n1(ctx->n1, K, nel, st);
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
