// The two other deposition operators of arXiv 2501.05340 on the affine periodic
// mesh (Sec. 2.3 deposition operator, Sec. 4.2 deposition), FP64-accurate:
//
//   corner nodes (IDW)  a particle at reference position xi of its element gives
//            q_c w_d(xi) to each corner d of the element, w_d(xi) = prod_a (1 -/+ xi_a)/2
//            (lower / upper corner per axis); a node's density is its sum over the
//            (periodic, unique) node divided by its volume V = sum over the elements
//            around it of sum_g W_g |J| w_d(xi_g); the field at a Gauss node is the
//            trilinear interpolation of the element's 8 corner densities.
//              k_idw_corner  one warp per element: the 8 x 4 corner sums over the
//                            element's particles (bin order), df32 -> corner[e][8][4]
//              k_idw_node    one thread per (node, component): the node's sum over
//                            the 8 elements around it in a fixed order, times 1/V
//              k_idw_field   one CTA per element: x and y passes of the trilinear
//                            interpolation in df32, then one FP64 FMA per output
//                            F = base(j,i) + hi_k (top(j,i) - base(j,i)).
// On GB300 one FP64 FMA (about 1.7 lanes per clock per SM) is cheaper than building
// a double from a df32 pair by integer operations (about 50 ALU operations at 64
// lanes per clock), so doubles are built by integer operations only where they are
// few (per element row, per node hit) and the per-output work is one FP64 FMA.
//   nearest DOF (Dirac) the whole source goes to the Gauss node nearest in reference
//            coordinates (per axis, the lower index on a tie) as q / (W_g |J|):
//              k_dirac       one warp per element: chunks of 32 particles mapped to
//                            their node, the lanes on one node summed by the first
//                            of them in bin order, each node hit scaled once, then
//                            the element's block of the field written from shared
//                            memory.
//
// FP64 arithmetic is kept off the per-particle and per-product paths: the reference
// coordinate comes from an exact fixed-point product of the position's bits, sums and
// products run in double-float (df32) on the FP32 pipe. Particles are binned by element first (pc_elem_bin: element, then id);
// every sum has a fixed order, so both results are deterministic; no atomics on data.
#include <math.h>
#include <string.h>

#include "pc_internal.cuh"

namespace {

constexpr int kCornerWarps = 8;  // elements per CTA of k_idw_corner
constexpr int kFieldThreads = 256;
constexpr unsigned long long kOne52 = 1ull << 52;
// Dirac: decisions closer than this (in units of 2^-52 of an element) to a node
// midpoint or an element face are taken again in FP64 exactly as the definition states.
constexpr long long kDiracMargin = 1ll << 12;

struct NodalArgs {
  int64_t n;
  int ne, n1;
  f2 lo[16], hi[16];         // (1 - eta_i)/2, (1 + eta_i)/2 (df32)
  double hi_d[16];           // (1 + eta_i)/2
  double eta[16];            // Gauss nodes
  f2 inv_wf[16];             // 1 / w_i (df32)
  f2 inv_jacf;               // (2/h)^3 (df32)
  unsigned long long mid[16];  // node midpoints ((eta_m + eta_m+1)/2 + 1)/2 in units of 2^-52
  double ne_d;
  f2 inv_vol;                // 1 / V
  const int32_t* start;
  const int32_t* perm;
  const double* x;
  const double* q;
  f2* corner;  // [nel][8][4] df32 corner sums
  f2* dens;    // [nel nodes][4] df32 node densities
  double* field;
};

// floor(x 2^52) for x in [0,1) from the bits of x (exact for x >= 1/2, the bits below
// 2^-52 dropped otherwise). Out-of-range values, which the binning reports as
// PC_EINVAL, are clamped so that every later index stays in range.
__device__ __forceinline__ unsigned long long fixed52(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  if (u >> 63) return 0;
  const int E = (int)((u >> 52) & 0x7FF);
  const int s = 1023 - E;  // x = (2^52 + M) 2^(E - 1075), so x 2^52 = (2^52 + M) >> (1023 - E)
  if (s <= 0) return kOne52 - 1;
  if (s > 53 || E == 0) return 0;
  return ((u & (kOne52 - 1)) | kOne52) >> s;
}

// Fraction x ne - ea of axis coordinate x inside element coordinate ea, in units of
// 2^-52 (signed: the binning rounds x ne, this product is exact).
__device__ __forceinline__ long long frac52(double x, int ne, int ea) {
  return (long long)(fixed52(x) * (unsigned long long)ne) - ((long long)ea << 52);
}

// v 2^-23 for an integer 0 <= v < 2^23, exactly, by (1 + v 2^-23) - 1 on the FP32 pipe
// (on GB300 the int-to-float conversions issue at the FP64 rate).
__device__ __forceinline__ float u23_scaled(unsigned v) { return __uint_as_float(0x3F800000u | v) - 1.0f; }

// A double as a normalised df32 pair by integer operations only, keeping 46 bits of
// the significand, for |v| in [2^-126, 2^128); smaller magnitudes give 0, larger
// ones infinity. (Every instruction of a predicated-off fallback would still occupy
// GB300's slow FP64 pipe, so there is no conversion path.)
__device__ __forceinline__ f2 split_f64(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(u >> 32);
  const int E = (int)((hi >> 20) & 0x7FF);
  const unsigned sign = hi & 0x80000000u;
  if (E < 897) return {__uint_as_float(sign), 0.0f};
  if (E > 1150) return {__uint_as_float(sign | 0x7F800000u), 0.0f};
  const float h = __uint_as_float(sign | ((unsigned)(E - 896) << 23) | (unsigned)((u >> 29) & 0x7FFFFFu));
  // significand bits 6..28 below h: their value is u23_scaled(bits) 2^(E - 1046), a
  // subnormal power of two for E < 920
  const unsigned sc = E >= 920 ? ((unsigned)(E - 919) << 23) : (1u << (E - 897));
  return fast_two_sum(h, u23_scaled((unsigned)(u >> 6) & 0x7FFFFFu) * __uint_as_float(sign | sc));
}

// Upper-corner factor f = (1 + xi)/2 = fr 2^-52 and lower-corner factor 1 - f of a
// fraction fr in [0, 2^52), as df32 pairs (46 bits; 1 - h is exact).
__device__ __forceinline__ void corner_factors(long long fr, f2* lo, f2* hi) {
  fr = fr < 0 ? 0 : (fr >= (long long)kOne52 ? (long long)kOne52 - 1 : fr);
  const float h = u23_scaled((unsigned)((unsigned long long)fr >> 29));
  const float l = u23_scaled((unsigned)(fr >> 6) & 0x7FFFFFu) * 1.1920928955078125e-07f;
  *hi = two_sum(h, l);
  *lo = two_sum(1.0f - h, -l);
}


// acc += a b in df32.
__device__ __forceinline__ void df_acc_mul(f2& acc, f2 a, f2 b) {
  f2 p = two_prod(a.h, b.h);
  p.l = fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
  f2 s = two_sum(acc.h, p.h);
  s.l = s.l + (acc.l + p.l);
  acc = fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ int wrap_idx(int a, int n) { return a >= n ? a - n : (a < 0 ? a + n : a); }

__global__ void __launch_bounds__(32 * kCornerWarps) k_idw_corner(const NodalArgs A, int nel) {
  __shared__ f2 sw[kCornerWarps][8][32];  // corner weights of the staged particles
  __shared__ f2 sq[kCornerWarps][4][32];  // their sources
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned e = blockIdx.x * kCornerWarps + wid;
  if (e >= (unsigned)nel) return;
  const unsigned ne = (unsigned)A.ne, r = e / ne;
  const int ea[3] = {(int)(e - r * ne), (int)(r % ne), (int)(r / ne)};
  const int d = lane >> 2, c = lane & 3;  // this lane's output: corner d, component c
  const int b = A.start[e], end = A.start[e + 1];
  // two independent chains (even and odd staged particles), joined in a fixed order
  f2 acc0 = {0.0f, 0.0f}, acc1 = {0.0f, 0.0f};
  for (int k0 = b; k0 < end; k0 += 32) {
    const int cnt = min(32, end - k0);
    if (lane < cnt) {
      const int i = A.perm[k0 + lane];
      f2 f[3][2];
#pragma unroll
      for (int a = 0; a < 3; ++a) corner_factors(frac52(A.x[a * A.n + i], A.ne, ea[a]), &f[a][0], &f[a][1]);
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const f2 fxy = df_mul(f[0][dx], f[1][dy]);
          sw[wid][2 * dy + dx][lane] = df_mul(fxy, f[2][0]);
          sw[wid][4 + 2 * dy + dx][lane] = df_mul(fxy, f[2][1]);
        }
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) sq[wid][cc][lane] = split_f64(A.q[cc * A.n + i]);
    }
    __syncwarp();
    int k = 0;
    for (; k + 1 < cnt; k += 2) {
      df_acc_mul(acc0, sq[wid][c][k], sw[wid][d][k]);
      df_acc_mul(acc1, sq[wid][c][k + 1], sw[wid][d][k + 1]);
    }
    if (k < cnt) df_acc_mul(acc0, sq[wid][c][k], sw[wid][d][k]);
    __syncwarp();
  }
  A.corner[(size_t)e * 32 + lane] = df_add(acc0, acc1);
}

// One thread per (node, component): the node's sum over the 8 elements around it, in
// which it is the corner opposite to the element's position, times 1/V.
__global__ void __launch_bounds__(256) k_idw_node(const NodalArgs A, int64_t nel) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * nel) return;
  const int ne = A.ne;
  const int64_t node = t >> 2;
  const int c = (int)(t & 3);
  const int nx = (int)(node % ne), ny = (int)((node / ne) % ne), nz = (int)(node / ((int64_t)ne * ne));
  f2 s = {0.0f, 0.0f};
  for (int a = 0; a < 8; ++a) {
    const int gx = wrap_idx(nx - 1 + (a & 1), ne), gy = wrap_idx(ny - 1 + ((a >> 1) & 1), ne),
              gz = wrap_idx(nz - 1 + (a >> 2), ne);
    const int64_t g = ((int64_t)gz * ne + gy) * ne + gx;
    s = df_add(s, A.corner[g * 32 + (7 - a) * 4 + c]);
  }
  A.dens[t] = df_mul(s, A.inv_vol);
}

template <int N1>
__global__ void __launch_bounds__(kFieldThreads) k_idw_field(const NodalArgs A) {
  constexpr int N2 = N1 * N1, NODES = N2 * N1;
  __shared__ f2 D[4][8];              // [component][corner] node densities
  __shared__ f2 ex[4][2][2][N1];      // x pass: [c][dz][dy][i]
  __shared__ double base[4][N2], slope[4][N2];  // y pass: [c][j N1 + i]
  const unsigned ne = (unsigned)A.ne, e = blockIdx.x, r = e / ne;
  const int ex0 = (int)(e - r * ne), ey0 = (int)(r % ne), ez0 = (int)(r / ne);
  const int t = threadIdx.x;
  if (t < 32) {
    const int d = t >> 2, c = t & 3;
    const int nx = wrap_idx(ex0 + (d & 1), A.ne), ny = wrap_idx(ey0 + ((d >> 1) & 1), A.ne),
              nz = wrap_idx(ez0 + (d >> 2), A.ne);
    D[c][d] = A.dens[(((size_t)nz * ne + ny) * ne + nx) * 4 + c];
  }
  __syncthreads();
  if (t < 16 * N1) {
    const int i = t % N1, rr = t / N1, c = rr & 3, dy = (rr >> 2) & 1, dz = rr >> 3;
    f2 s = df_mul(A.lo[i], D[c][4 * dz + 2 * dy]);
    df_acc_mul(s, A.hi[i], D[c][4 * dz + 2 * dy + 1]);
    ex[c][dz][dy][i] = s;
  }
  __syncthreads();
  for (int o = t; o < 4 * N2; o += kFieldThreads) {
    const int c = o / N2, ji = o % N2, j = ji / N1, i = ji % N1;
    f2 b0 = df_mul(A.lo[j], ex[c][0][0][i]);
    df_acc_mul(b0, A.hi[j], ex[c][0][1][i]);
    f2 b1 = df_mul(A.lo[j], ex[c][1][0][i]);
    df_acc_mul(b1, A.hi[j], ex[c][1][1][i]);
    base[c][ji] = df_to_f64(b0);
    slope[c][ji] = df_to_f64(df_add(b1, df_neg(b0)));
  }
  __syncthreads();
  // z pass: one FP64 FMA per output (cheaper on GB300 than building a double from a
  // df32 pair by integer operations), streaming stores
  double* out = A.field + (size_t)e * 4 * NODES;
  for (int o = t; o < 4 * NODES; o += kFieldThreads) {
    const int c = o / NODES, g = o % NODES, k = g / N2, ji = g % N2;
    __stcs(out + o, __fma_rn(A.hi_d[k], slope[c][ji], base[c][ji]));
  }
}

// Nearest node index along one axis exactly as the definition states: FP64 reference
// coordinate 2 (x ne - e) - 1, argmin |eta_m - xi| with the lower index on a tie.
__device__ __forceinline__ int nearest_fp64(const NodalArgs& A, double y) {
  const double t = __dmul_rn(y, A.ne_d);
  int e = (int)floor(t);
  e = e < 0 ? 0 : (e > A.ne - 1 ? A.ne - 1 : e);
  const double xi = __dsub_rn(__dmul_rn(2.0, __dsub_rn(t, (double)e)), 1.0);
  int best = 0;
  double bd = fabs(A.eta[0] - xi);
  for (int m = 1; m < A.n1; ++m) {
    const double dm = fabs(A.eta[m] - xi);
    if (dm < bd) {
      bd = dm;
      best = m;
    }
  }
  return best;
}

// Shared memory of k_dirac per warp (one element): the df32 node sums [4][NODES]
// (later the doubles of the field block), the staged sources [4][32], the list of
// nodes hit and a flag byte per node; 16-byte multiples.
template <int N1>
struct DiracShape {
  static constexpr int NODES = N1 * N1 * N1;
  static constexpr int LIST = (NODES + 3) & ~3;
  static constexpr int FLAGS = (NODES + 15) & ~15;
  static constexpr size_t PER_WARP = (size_t)4 * NODES * sizeof(f2) + 4 * 32 * sizeof(f2) + LIST * sizeof(int) + FLAGS;
  static constexpr int WARPS = PER_WARP * 4 <= 98304 ? 4 : (PER_WARP * 2 <= 98304 ? 2 : 1);
  static constexpr size_t SMEM = PER_WARP * WARPS;
};

// One warp per element: chunks of 32 particles in bin order; the lanes on the same
// node (__match_any_sync) are summed by the lowest of them in lane order and added to
// the node's sum, so every sum has the bin order.
template <int N1>
__global__ void __launch_bounds__(32 * DiracShape<N1>::WARPS) k_dirac(const NodalArgs A, int nel) {
  using S = DiracShape<N1>;
  constexpr int NODES = S::NODES;
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned e = blockIdx.x * S::WARPS + wid;
  if (e >= (unsigned)nel) return;
  f2* acc = reinterpret_cast<f2*>(dsm_raw + wid * S::PER_WARP);  // [4][NODES]
  f2* sq = acc + 4 * NODES;                                       // [4][32]
  int* list = reinterpret_cast<int*>(sq + 4 * 32);                // [LIST]
  unsigned char* flag = reinterpret_cast<unsigned char*>(list + S::LIST);
  for (int o = lane; o < 2 * NODES; o += 32) reinterpret_cast<float4*>(acc)[o] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int o = lane; o < S::FLAGS / 4; o += 32) reinterpret_cast<unsigned*>(flag)[o] = 0u;
  const unsigned ne = (unsigned)A.ne, r = e / ne;
  const int ea[3] = {(int)(e - r * ne), (int)(r % ne), (int)(r / ne)};
  const int b = A.start[e], end = A.start[e + 1];
  int nlist = 0;
  __syncwarp();
  for (int k0 = b; k0 < end; k0 += 32) {
    const int cnt = min(32, end - k0);
    const bool act = lane < cnt;
    int g = -1 - lane;  // distinct for idle lanes
    if (act) {
      const int i = A.perm[k0 + lane];
      g = 0;
#pragma unroll
      for (int a = 2; a >= 0; --a) {
        const double y = A.x[a * A.n + i];
        const long long f = frac52(y, A.ne, ea[a]);
        bool sure = f >= kDiracMargin && f < (long long)kOne52 - kDiracMargin;
        int m = 0;
#pragma unroll
        for (int q = 0; q + 1 < N1; ++q) {
          const long long dm = f - (long long)A.mid[q];
          sure = sure && (dm > kDiracMargin || dm < -kDiracMargin);
          m += dm > 0;
        }
        // the FP64 decision behind a warp-uniform branch, so that it is never issued
        // predicated off
        if (__any_sync(__activemask(), !sure))
          if (!sure) m = nearest_fp64(A, y);
        g = g * N1 + m;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) sq[c * 32 + lane] = split_f64(A.q[c * A.n + i]);
    }
    __syncwarp();
    const unsigned grp = __match_any_sync(0xffffffffu, g);
    const bool leader = act && (__ffs(grp) - 1 == lane);
    if (leader) {
      f2 s[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) s[c] = sq[c * 32 + lane];
      for (unsigned m = grp & (grp - 1); m; m &= m - 1) {
        const int k = __ffs(m) - 1;
#pragma unroll
        for (int c = 0; c < 4; ++c) s[c] = df_add(s[c], sq[c * 32 + k]);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c * NODES + g] = df_add(acc[c * NODES + g], s[c]);
    }
    const bool fresh = leader && !flag[g];
    const unsigned fm = __ballot_sync(0xffffffffu, fresh);
    if (fresh) {
      flag[g] = 1;
      list[nlist + __popc(fm & ((1u << lane) - 1u))] = g;
    }
    nlist += __popc(fm);
    __syncwarp();
  }
  // densities of the nodes hit, written over their sums as doubles
  for (int rr = lane; rr < nlist; rr += 32) {
    const int g = list[rr];
    const int i = g % N1, j = (g / N1) % N1, k = g / (N1 * N1);
    const f2 iw = df_mul(df_mul(df_mul(A.inv_wf[i], A.inv_wf[j]), A.inv_wf[k]), A.inv_jacf);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double v = df_to_f64(df_mul(acc[c * NODES + g], iw));
      acc[c * NODES + g] = *reinterpret_cast<const f2*>(&v);
    }
  }
  __syncwarp();
  double2* out = reinterpret_cast<double2*>(A.field + (size_t)e * 4 * NODES);
  for (int o = lane; o < 2 * NODES; o += 32) __stcs(out + o, reinterpret_cast<const double2*>(acc)[o]);
}

template <int N1>
cudaError_t launch_nodal(bool dirac, const NodalArgs& A, unsigned nel, cudaStream_t st) {
  if (dirac) {
    using S = DiracShape<N1>;
    PC_CUDA_TRY(cudaFuncSetAttribute(k_dirac<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM));
    k_dirac<N1><<<(nel + S::WARPS - 1) / S::WARPS, 32 * S::WARPS, S::SMEM, st>>>(A, (int)nel);
  } else {
    k_idw_field<N1><<<nel, kFieldThreads, 0, st>>>(A);
  }
  return cudaGetLastError();
}

cudaError_t launch_nodal_n1(int n1, bool dirac, const NodalArgs& A, unsigned nel, cudaStream_t st) {
  switch (n1) {
#define PC_NODAL_CASE(N) \
  case N:                \
    return launch_nodal<N>(dirac, A, nel, st);
    PC_NODAL_CASE(1) PC_NODAL_CASE(2) PC_NODAL_CASE(3) PC_NODAL_CASE(4) PC_NODAL_CASE(5) PC_NODAL_CASE(6)
    PC_NODAL_CASE(7) PC_NODAL_CASE(8) PC_NODAL_CASE(9) PC_NODAL_CASE(10) PC_NODAL_CASE(11) PC_NODAL_CASE(12)
    PC_NODAL_CASE(13) PC_NODAL_CASE(14) PC_NODAL_CASE(15) PC_NODAL_CASE(16)
#undef PC_NODAL_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

f2 host_df(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

void fill_args(pc_ctx* ctx, const pc_particles* p, double* field, NodalArgs* A) {
  memset(A, 0, sizeof(*A));
  const int n1 = ctx->n1;
  A->n = p->n;
  A->ne = ctx->cfg.ne;
  A->n1 = n1;
  A->ne_d = (double)ctx->cfg.ne;
  const double h = 1.0 / (double)ctx->cfg.ne, jac = 0.125 * h * h * h;
  A->inv_jacf = host_df(8.0 * (double)ctx->cfg.ne * ctx->cfg.ne * ctx->cfg.ne);
  double lo[16], hi[16];
  for (int i = 0; i < n1; ++i) {
    lo[i] = 0.5 * (1.0 - ctx->eta[i]);
    hi[i] = 0.5 * (1.0 + ctx->eta[i]);
    A->lo[i] = host_df(lo[i]);
    A->hi[i] = host_df(hi[i]);
    A->hi_d[i] = hi[i];
    A->eta[i] = ctx->eta[i];
    A->inv_wf[i] = host_df(1.0 / ctx->w[i]);
  }
  for (int m = 0; m + 1 < n1; ++m) {
    const double mid = 0.5 * (0.5 * (ctx->eta[m] + ctx->eta[m + 1]) + 1.0);
    A->mid[m] = (unsigned long long)llround(ldexp(mid, 52));
  }
  // V: every node of the affine periodic mesh has 8 elements around it, where it is
  // each of the 8 corners once, so V = sum over corners d of sum_g W_g |J| w_d(xi_g)
  double vol = 0.0;
  for (int d = 0; d < 8; ++d)
    for (int k = 0; k < n1; ++k)
      for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n1; ++i) {
          const double fx = (d & 1) ? hi[i] : lo[i];
          const double fy = ((d >> 1) & 1) ? hi[j] : lo[j];
          const double fz = (d >> 2) ? hi[k] : lo[k];
          vol += ctx->w[i] * ctx->w[j] * ctx->w[k] * jac * (fx * fy * fz);
        }
  A->inv_vol = host_df(1.0 / vol);
  A->start = ctx->start;
  A->perm = ctx->perm;
  A->x = p->x;
  A->q = p->q;
  A->corner = reinterpret_cast<f2*>(ctx->corner);
  A->dens = A->corner + 32 * (int64_t)ctx->cfg.ne * ctx->cfg.ne * ctx->cfg.ne;
  A->field = field;
}

}  // namespace

pc_status pc_project_idw_impl(pc_ctx* ctx, const pc_particles* p, double* field) {
  const int ne = ctx->cfg.ne;
  const unsigned nel = (unsigned)ne * ne * ne;
  cudaStream_t st = ctx->stream;
  cudaError_t e = pc_elem_bin(ctx, p->n, p->x, p->id);
  if (e == cudaSuccess) {
    NodalArgs A;
    fill_args(ctx, p, field, &A);
    const int td = pc_phase_begin(ctx, PC_PH_DEPOSIT);
    k_idw_corner<<<(nel + kCornerWarps - 1) / kCornerWarps, 32 * kCornerWarps, 0, st>>>(A, (int)nel);
    k_idw_node<<<(4 * nel + 255) / 256, 256, 0, st>>>(A, (int64_t)nel);
    e = launch_nodal_n1(ctx->n1, false, A, nel, st);
    ctx->launches += 3;
    pc_phase_end(ctx, td);
  }
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_project_idw: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}

pc_status pc_project_dirac_impl(pc_ctx* ctx, const pc_particles* p, double* field) {
  const int ne = ctx->cfg.ne;
  const unsigned nel = (unsigned)ne * ne * ne;
  cudaStream_t st = ctx->stream;
  cudaError_t e = pc_elem_bin(ctx, p->n, p->x, p->id);
  if (e == cudaSuccess) {
    NodalArgs A;
    fill_args(ctx, p, field, &A);
    const int td = pc_phase_begin(ctx, PC_PH_DEPOSIT);
    e = launch_nodal_n1(ctx->n1, true, A, nel, st);
    ctx->launches += 1;
    pc_phase_end(ctx, td);
  }
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_project_dirac: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}
