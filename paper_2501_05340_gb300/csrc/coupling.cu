// Fluid -> particle coupling of arXiv 2501.05340 on the affine periodic mesh:
//
//   field evaluation (Sec. 3.2)   U(x_p) = sum_{ijk} U_ijk l_i(xi_1) l_j(xi_2) l_k(xi_3), l the Lagrange
//                                 basis of the Legendre-Gauss nodes, xi the particle's reference position
//                                 in its element. k_eval_field<N1>: one warp per element (particles binned
//                                 by element), the element's coefficients of one variable at a time in
//                                 shared memory as double-float pairs, one lane per particle; the basis by
//                                 prefix and suffix products of (xi - eta_m) and the contraction by sum
//                                 factorisation (i, then j, then k), all in double-float on the FP32 pipe.
//   drag sources (Sec. 2.2, 2.3)  F = 3 pi mu_f d f_D (u_f - v_p), f_D = 1 + 0.15 Re^0.687 (Schiller-Naumann;
//                                 the paper's correlation is not printed), q = (-F, -F.v_p):
//                                 k_drag_sources, one thread per particle, FP64.
//
// The reference coordinate comes from an exact fixed-point product of the position's bits,
// as in the nodal depositions; doubles are built from double-float pairs by integer
// operations (never-taken FP64 fallbacks would still occupy GB300's slow FP64 pipe).
#include <math.h>
#include <string.h>

#include "pc_internal.cuh"

namespace {

constexpr unsigned long long kOne52 = 1ull << 52;

struct EvalArgs {
  int64_t n;
  int ne, nvar;
  f2 eta[16];      // Gauss nodes (df32)
  f2 inv_den[16];  // 1 / prod_{m != i} (eta_i - eta_m) (df32)
  const int32_t* start;
  const int32_t* perm;
  const double* x;
  const double* field;  // [nel][nvar][N1^3]
  double* out;          // [nvar][n], input order
};

__device__ __forceinline__ float u23_scaled(unsigned v) { return __uint_as_float(0x3F800000u | v) - 1.0f; }

__device__ __forceinline__ unsigned long long fixed52(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  if (u >> 63) return 0;
  const int E = (int)((u >> 52) & 0x7FF);
  const int s = 1023 - E;
  if (s <= 0) return kOne52 - 1;
  if (s > 53 || E == 0) return 0;
  return ((u & (kOne52 - 1)) | kOne52) >> s;
}

// Reference coordinate 2 (x ne - ea) - 1 in [-1, 1) as a df32 pair from the exact
// fixed-point fraction fr 2^-52 (clamped to the element): with h = (fr >> 29) 2^-23 and
// l the next 23 bits, 2h - 1 is exact in FP32.
__device__ __forceinline__ f2 ref_coord(double x, int ne, int ea) {
  long long fr = (long long)(fixed52(x) * (unsigned long long)ne) - ((long long)ea << 52);
  fr = fr < 0 ? 0 : (fr >= (long long)kOne52 ? (long long)kOne52 - 1 : fr);
  const float h = u23_scaled((unsigned)((unsigned long long)fr >> 29));
  const float l = u23_scaled((unsigned)(fr >> 6) & 0x7FFFFFu) * 1.1920928955078125e-07f;
  return two_sum(2.0f * h - 1.0f, 2.0f * l);
}

__device__ __forceinline__ f2 split_f64(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(u >> 32);
  const int E = (int)((hi >> 20) & 0x7FF);
  const unsigned sign = hi & 0x80000000u;
  if (E < 897) return {__uint_as_float(sign), 0.0f};
  if (E > 1150) return {__uint_as_float(sign | 0x7F800000u), 0.0f};
  const float h = __uint_as_float(sign | ((unsigned)(E - 896) << 23) | (unsigned)((u >> 29) & 0x7FFFFFu));
  const unsigned sc = E >= 920 ? ((unsigned)(E - 919) << 23) : (1u << (E - 897));
  return fast_two_sum(h, u23_scaled((unsigned)(u >> 6) & 0x7FFFFFu) * __uint_as_float(sign | sc));
}


__device__ __forceinline__ void df_acc_mul(f2& acc, f2 a, f2 b) {
  f2 p = two_prod(a.h, b.h);
  p.l = fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
  f2 s = two_sum(acc.h, p.h);
  s.l = s.l + (acc.l + p.l);
  acc = fast_two_sum(s.h, s.l);
}

// Lagrange basis l_0..l_{N1-1} at xi: (prefix product of (xi - eta_m), m < i) times
// (suffix product, m > i) times 1 / prod (eta_i - eta_m).
template <int N1>
__device__ __forceinline__ void lagrange_basis(const EvalArgs& A, f2 xi, f2* l) {
  f2 d[N1], pre = {1.0f, 0.0f};
#pragma unroll
  for (int m = 0; m < N1; ++m) d[m] = df_add(xi, df_neg(A.eta[m]));
#pragma unroll
  for (int i = 0; i < N1; ++i) {
    l[i] = pre;
    pre = df_mul(pre, d[i]);
  }
  f2 suf = {1.0f, 0.0f};
#pragma unroll
  for (int i = N1 - 1; i >= 0; --i) {
    l[i] = df_mul(df_mul(l[i], suf), A.inv_den[i]);
    suf = df_mul(suf, d[i]);
  }
}

// Warps (elements) per CTA of k_eval_field: as many as fit 48 KB of static shared memory, at most 4.
template <int N1>
struct EvalShape {
  static constexpr int NODES = N1 * N1 * N1;
  static constexpr int PER_WARP = (NODES + 3 * N1 * 32) * (int)sizeof(f2);
  static constexpr int WARPS = 48000 / PER_WARP >= 4 ? 4 : (48000 / PER_WARP >= 2 ? 2 : 1);
};

template <int N1>
__global__ void __launch_bounds__(32 * EvalShape<N1>::WARPS) k_eval_field(const EvalArgs A, int nel) {
  constexpr int NODES = N1 * N1 * N1, W = EvalShape<N1>::WARPS;
  __shared__ f2 su[W][NODES];          // one variable of the element's coefficients
  __shared__ f2 sb[W][3][N1][32];      // the staged particles' basis values per axis
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned e = blockIdx.x * W + wid;
  if (e >= (unsigned)nel) return;
  const unsigned ne = (unsigned)A.ne, r = e / ne;
  const int ea[3] = {(int)(e - r * ne), (int)(r % ne), (int)(r / ne)};
  const int b = A.start[e], end = A.start[e + 1];
  if (b == end) return;
  const double* U = A.field + (size_t)e * A.nvar * NODES;
  for (int k0 = b; k0 < end; k0 += 32) {
    const int cnt = min(32, end - k0);
    int p = 0;
    if (lane < cnt) {
      p = A.perm[k0 + lane];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        f2 l[N1];
        lagrange_basis<N1>(A, ref_coord(A.x[a * A.n + p], A.ne, ea[a]), l);
#pragma unroll
        for (int i = 0; i < N1; ++i) sb[wid][a][i][lane] = l[i];
      }
    }
    for (int c = 0; c < A.nvar; ++c) {
      __syncwarp();
      for (int g = lane; g < NODES; g += 32) su[wid][g] = split_f64(U[c * NODES + g]);
      __syncwarp();
      if (lane < cnt) {
        f2 val = {0.0f, 0.0f};
        for (int k = 0; k < N1; ++k) {
          f2 sk = {0.0f, 0.0f};
          for (int j = 0; j < N1; ++j) {
            f2 sj = {0.0f, 0.0f};
#pragma unroll
            for (int i = 0; i < N1; ++i) df_acc_mul(sj, sb[wid][0][i][lane], su[wid][(k * N1 + j) * N1 + i]);
            df_acc_mul(sk, sb[wid][1][j][lane], sj);
          }
          df_acc_mul(val, sb[wid][2][k][lane], sk);
        }
        A.out[(size_t)c * A.n + p] = df_to_f64(val);
      }
    }
    __syncwarp();
  }
}

template <int N1>
cudaError_t launch_eval(const EvalArgs& A, unsigned nel, cudaStream_t st) {
  constexpr int W = EvalShape<N1>::WARPS;
  k_eval_field<N1><<<(nel + W - 1) / W, 32 * W, 0, st>>>(A, (int)nel);
  return cudaGetLastError();
}

cudaError_t launch_eval_n1(int n1, const EvalArgs& A, unsigned nel, cudaStream_t st) {
  switch (n1) {
#define PC_EVAL_CASE(N) \
  case N:               \
    return launch_eval<N>(A, nel, st);
    PC_EVAL_CASE(1) PC_EVAL_CASE(2) PC_EVAL_CASE(3) PC_EVAL_CASE(4) PC_EVAL_CASE(5) PC_EVAL_CASE(6)
    PC_EVAL_CASE(7) PC_EVAL_CASE(8) PC_EVAL_CASE(9) PC_EVAL_CASE(10) PC_EVAL_CASE(11) PC_EVAL_CASE(12)
    PC_EVAL_CASE(13) PC_EVAL_CASE(14) PC_EVAL_CASE(15) PC_EVAL_CASE(16)
#undef PC_EVAL_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

// Drag force and its sources per particle, FP64 in the written order.
__global__ void k_drag_sources(int64_t n, const double* __restrict__ v, const double* __restrict__ r,
                               const double* __restrict__ fluid, double mu_f, double* __restrict__ q) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double pi = 3.14159265358979323846;
  const double d = 2.0 * r[p];
  const double rho = fluid[p];
  const double vp[3] = {v[p], v[n + p], v[2 * n + p]};
  double rel[3], F[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) rel[k] = fluid[(k + 1) * n + p] - vp[k];
  const double speed = sqrt((rel[0] * rel[0] + rel[1] * rel[1]) + rel[2] * rel[2]);
  const double re = rho * speed * d / mu_f;
  const double fd = 1.0 + 0.15 * pow(re, 0.687);
  const double coef = 3.0 * pi * mu_f * d * fd;
#pragma unroll
  for (int k = 0; k < 3; ++k) F[k] = coef * rel[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) q[k * n + p] = -F[k];
  q[3 * n + p] = -((F[0] * vp[0] + F[1] * vp[1]) + F[2] * vp[2]);
}

f2 host_df(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

}  // namespace

pc_status pc_eval_field_impl(pc_ctx* ctx, const pc_particles* p, const double* field, int nvar, double* out) {
  const int ne = ctx->cfg.ne, n1 = ctx->n1;
  const unsigned nel = (unsigned)ne * ne * ne;
  cudaError_t e = pc_elem_bin(ctx, p->n, p->x, p->id);
  if (e == cudaSuccess && p->n > 0) {
    EvalArgs A;
    memset(&A, 0, sizeof(A));
    A.n = p->n;
    A.ne = ne;
    A.nvar = nvar;
    for (int i = 0; i < n1; ++i) {
      double den = 1.0;
      for (int m = 0; m < n1; ++m)
        if (m != i) den *= ctx->eta[i] - ctx->eta[m];
      A.eta[i] = host_df(ctx->eta[i]);
      A.inv_den[i] = host_df(1.0 / den);
    }
    A.start = ctx->start;
    A.perm = ctx->perm;
    A.x = p->x;
    A.field = field;
    A.out = out;
    const int td = pc_phase_begin(ctx, PC_PH_DEPOSIT);
    e = launch_eval_n1(n1, A, nel, ctx->stream);
    ctx->launches += 1;
    pc_phase_end(ctx, td);
  }
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_eval_field: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}

pc_status pc_drag_sources_impl(pc_ctx* ctx, const pc_particles* p, const double* fluid, double mu_f, double* q) {
  if (p->n > 0) {
    k_drag_sources<<<pc_blocks(p->n, 256), 256, 0, ctx->stream>>>(p->n, p->v, p->r, fluid, mu_f, q);
    ctx->launches += 1;
  }
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_drag_sources: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}
