// Differentiation of the particle operator with the pair set held fixed: replay of
// a step with a given matching, and the vector-Jacobian products of the step and
// of the projection. (Not in the paper; used for differentiable rollouts.)
//
// Compiled with -fmad=false: the replay evaluates the same IEEE operations in the
// same order as pc_collide, so it is bit-identical for the same pair set.
#include <math.h>

#include "pc_internal.cuh"

namespace {

__device__ __forceinline__ double minimg(double d) {
  if (d > 0.5) return d - 1.0;
  if (d < -0.5) return d + 1.0;
  return d;
}

__device__ __forceinline__ double wrap01(double y) {
  double w = y - floor(y);
  if (w == 1.0) w = 0.0;
  return w;
}

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

__device__ __forceinline__ int cell_of(double y, int nc) {
  int c = (int)(y * (double)nc);
  c = c < 0 ? 0 : c;
  return c >= nc ? nc - 1 : c;
}

__device__ __forceinline__ double dot3(const double a[3], const double b[3]) {
  return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

// Contact time of the pair (i, j) from i's side (same sequence as pc_collide).
__device__ double pair_time(const double xi[3], const double xj[3], const double vi[3], const double vj[3],
                            double R, double dt) {
  double dx[3], dv[3];
  for (int a = 0; a < 3; ++a) {
    dx[a] = minimg(xi[a] - xj[a]);
    dv[a] = vi[a] - vj[a];
  }
  const double a = (dv[0] * dv[0] + dv[1] * dv[1]) + dv[2] * dv[2];
  const double b = (dx[0] * dv[0] + dx[1] * dv[1]) + dx[2] * dv[2];
  const double c = ((dx[0] * dx[0] + dx[1] * dx[1]) + dx[2] * dx[2]) - R * R;
  if (!(b < 0.0)) return CUDART_INF;
  if (!(c > 0.0)) return CUDART_INF;
  const double disc = b * b - a * c;
  if (!(disc > 0.0)) return CUDART_INF;
  const double t = c / (-b + sqrt(disc));
  return t <= dt ? t : CUDART_INF;
}

__global__ void k_pairs_to_partner(int64_t n_ids, const unsigned long long* __restrict__ counters,
                                   const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                   int32_t* __restrict__ partner) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t np = (int64_t)counters[CNT_PAIRS];
  if (i < np) {
    const int32_t a = lo[i], b = hi[i];
    if (a >= 0 && a < n_ids && b >= 0 && b < n_ids) {
      partner[a] = b;
      partner[b] = a;
    } else {
      atomicMax((unsigned long long*)&counters[CNT_STATUS], (unsigned long long)PC_EINVAL);
    }
  }
}

struct ReplayArgs {
  int64_t n;
  double dt, e;
  const double *x, *v, *r, *m, *q;
  const int32_t* id;
  const int32_t* partner;
  double *xo, *vo, *ro, *mo, *qo;
  int32_t* ido;
  unsigned long long* counters;
};

// The replayed pair step of particle i (partner j): contact time, response, advance;
// a pair without a root in [0, dt] is recorded as PC_EREPLAY and flies free.
__device__ __forceinline__ void replay_pair(const ReplayArgs& A, int64_t i, int32_t j) {
  const int64_t n = A.n;
  const double xi[3] = {A.x[i], A.x[n + i], A.x[2 * n + i]};
  const double vi[3] = {A.v[i], A.v[n + i], A.v[2 * n + i]};
  double xo[3], vo[3];
  const double xj[3] = {A.x[j], A.x[n + j], A.x[2 * n + j]};
  const double vj[3] = {A.v[j], A.v[n + j], A.v[2 * n + j]};
  const double t = pair_time(xi, xj, vi, vj, A.r[i] + A.r[j], A.dt);
  if (!(t <= A.dt)) {
    atomicMax(&A.counters[CNT_STATUS], (unsigned long long)PC_EREPLAY);
    for (int a = 0; a < 3; ++a) {
      vo[a] = vi[a];
      xo[a] = xi[a] + A.dt * vi[a];
    }
  } else {
    double dx[3], dv[3], s[3], nr[3];
    for (int a = 0; a < 3; ++a) {
      dx[a] = minimg(xi[a] - xj[a]);
      dv[a] = vi[a] - vj[a];
    }
    for (int a = 0; a < 3; ++a) s[a] = dx[a] + t * dv[a];
    const double sl = sqrt((s[0] * s[0] + s[1] * s[1]) + s[2] * s[2]);
    for (int a = 0; a < 3; ++a) nr[a] = -s[a] / sl;
    const double vrn = (dv[0] * nr[0] + dv[1] * nr[1]) + dv[2] * nr[2];
    const double mi = A.m[i], mj = A.m[j];
    const double mr = (mi * mj) / (mi + mj);
    const double J = -mr * (1.0 + A.e) * vrn;
    const double gi = J / mi;
    for (int a = 0; a < 3; ++a) {
      const double vnew = vi[a] + gi * nr[a];
      vo[a] = vnew;
      xo[a] = (xi[a] + t * vi[a]) + (A.dt - t) * vnew;
    }
  }
  for (int a = 0; a < 3; ++a) {
    A.xo[a * n + i] = wrap01(xo[a]);
    A.vo[a * n + i] = vo[a];
  }
}

// One thread per particle for free flight and the copies; the block's colliding
// particles are queued and replayed by the block's first threads together (an FP64
// instruction takes a warp the same pipe time whatever the number of active lanes).
__global__ void __launch_bounds__(256) k_replay(ReplayArgs A) {
  __shared__ int q_cnt;
  __shared__ int q_i[256];
  if (threadIdx.x == 0) q_cnt = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  if (i < n) {
    if (A.partner[i] < 0) {
      for (int a = 0; a < 3; ++a) {
        const double vi = A.v[a * n + i];
        A.xo[a * n + i] = wrap01(A.x[a * n + i] + A.dt * vi);
        A.vo[a * n + i] = vi;
      }
    } else {
      q_i[atomicAdd(&q_cnt, 1)] = threadIdx.x;
    }
    if (A.ro) A.ro[i] = A.r[i];
    if (A.mo) A.mo[i] = A.m[i];
    if (A.ido) A.ido[i] = A.id[i];
    if (A.qo)
      for (int c = 0; c < 4; ++c) A.qo[c * n + i] = A.q[c * n + i];
  }
  __syncthreads();
  const int nq = q_cnt;
  for (int e = threadIdx.x; e < nq; e += blockDim.x) {
    const int64_t ii = (int64_t)blockIdx.x * blockDim.x + q_i[e];
    replay_pair(A, ii, A.partner[ii]);
  }
}

struct AdjArgs {
  int64_t n;
  double dt, e;
  const double *x, *v, *r, *m;
  const int32_t* partner;
  const double *gxo, *gvo;
  double *gxi, *gvi;
  unsigned long long* counters;
};

// Reverse sweep of one pair's response, from particle i's side; writes i's cotangents.
// Forward: t from |dx + t dv| = R, s = dx + t dv, n = -s/|s|, J = -m_r (1+e) dv.n,
// v_i' = v_i + (J/m_i) n, v_j' = v_j - (J/m_j) n, x_k' = x_k + t v_k + (dt - t) v_k'.
__device__ __forceinline__ void adjoint_pair(const AdjArgs& A, int64_t i, int32_t j) {
  const int64_t n = A.n;
  const double xi[3] = {A.x[i], A.x[n + i], A.x[2 * n + i]};
  const double vi[3] = {A.v[i], A.v[n + i], A.v[2 * n + i]};
  const double xj[3] = {A.x[j], A.x[n + j], A.x[2 * n + j]};
  const double vj[3] = {A.v[j], A.v[n + j], A.v[2 * n + j]};
  const double t = pair_time(xi, xj, vi, vj, A.r[i] + A.r[j], A.dt);
  if (!(t <= A.dt)) {
    atomicMax(&A.counters[CNT_STATUS], (unsigned long long)PC_EREPLAY);
    for (int a = 0; a < 3; ++a) {
      A.gxi[a * n + i] = 0.0;
      A.gvi[a * n + i] = 0.0;
    }
    return;
  }
  const double mi = A.m[i], mj = A.m[j];
  double dx[3], dv[3], s[3], nr[3], vin[3], vjn[3];
  for (int a = 0; a < 3; ++a) {
    dx[a] = minimg(xi[a] - xj[a]);
    dv[a] = vi[a] - vj[a];
    s[a] = dx[a] + t * dv[a];
  }
  const double sl = sqrt(dot3(s, s));
  for (int a = 0; a < 3; ++a) nr[a] = -s[a] / sl;
  const double vrn = dot3(dv, nr);
  const double mr = (mi * mj) / (mi + mj);
  const double J = -mr * (1.0 + A.e) * vrn;
  for (int a = 0; a < 3; ++a) {
    vin[a] = vi[a] + (J / mi) * nr[a];
    vjn[a] = vj[a] - (J / mj) * nr[a];
  }
  double Vit[3], Vjt[3], gn[3] = {0, 0, 0}, gdv[3] = {0, 0, 0}, gdx[3] = {0, 0, 0}, gvi_own[3];
  double gt = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double Xi = A.gxo[a * n + i], Xj = A.gxo[a * n + j];
    gvi_own[a] = t * Xi;
    Vit[a] = A.gvo[a * n + i] + (A.dt - t) * Xi;
    Vjt[a] = A.gvo[a * n + j] + (A.dt - t) * Xj;
    gt += Xi * (vi[a] - vin[a]) + Xj * (vj[a] - vjn[a]);
  }
  for (int a = 0; a < 3; ++a) {
    gvi_own[a] += Vit[a];
    gn[a] += (J / mi) * Vit[a] - (J / mj) * Vjt[a];
  }
  const double gJ = dot3(Vit, nr) / mi - dot3(Vjt, nr) / mj;
  const double gvrn = -mr * (1.0 + A.e) * gJ;
  for (int a = 0; a < 3; ++a) {
    gdv[a] += gvrn * nr[a];
    gn[a] += gvrn * dv[a];
  }
  const double nh[3] = {s[0] / sl, s[1] / sl, s[2] / sl};
  const double pg = dot3(nh, gn);
  double gs[3];
  for (int a = 0; a < 3; ++a) gs[a] = -(gn[a] - nh[a] * pg) / sl;
  for (int a = 0; a < 3; ++a) {
    gdx[a] += gs[a];
    gdv[a] += t * gs[a];
  }
  gt += dot3(gs, dv);
  const double sdv = dot3(s, dv);
  for (int a = 0; a < 3; ++a) {
    gdx[a] += gt * (-s[a] / sdv);
    gdv[a] += gt * (-t * s[a] / sdv);
  }
  for (int a = 0; a < 3; ++a) {
    A.gxi[a * n + i] = A.gxo[a * n + i] + gdx[a];
    A.gvi[a * n + i] = gvi_own[a] + gdv[a];
  }
}

// One thread per particle for the free ones; the block's colliding particles are
// queued and swept by the block's first threads together, as in k_replay.
__global__ void __launch_bounds__(256) k_collide_adjoint(AdjArgs A) {
  __shared__ int q_cnt;
  __shared__ int q_i[256];
  if (threadIdx.x == 0) q_cnt = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  if (i < n) {
    if (A.partner[i] < 0) {
      for (int a = 0; a < 3; ++a) {
        A.gxi[a * n + i] = A.gxo[a * n + i];
        A.gvi[a * n + i] = A.gvo[a * n + i] + A.dt * A.gxo[a * n + i];
      }
    } else {
      q_i[atomicAdd(&q_cnt, 1)] = threadIdx.x;
    }
  }
  __syncthreads();
  const int nq = q_cnt;
  for (int e = threadIdx.x; e < nq; e += blockDim.x) {
    const int64_t ii = (int64_t)blockIdx.x * blockDim.x + q_i[e];
    adjoint_pair(A, ii, A.partner[ii]);
  }
}

struct ProjAdjArgs {
  int64_t n;
  int ne, n1, rho, win;
  double h, rc, inv2s2, inv_s2, scale;  // scale = (2/h)^3
  double eta[16], w[16];
  const double *x, *q, *G;
  double *gq, *gx;
};

// One warp per particle (in the caller's order): the window factors k_a and
// offsets d = X - x on its own element and rho neighbours per axis, Z_a, the
// weighted mean offsets mu_a, then a sweep over the support box reading G:
//   gq_c = (2/h)^3 sum_g G_gc khat, gx_a = (2/h)^3 / sigma^2 sum_g a_g khat (d_a - mu_a),
// with a_g = sum_c G_gc q_c and khat = kx ky kz / (Zx Zy Zz).
__global__ void __launch_bounds__(128) k_project_adjoint(ProjAdjArgs A) {
  __shared__ double kf[4][3][64];
  __shared__ double dd[4][3][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * 4 + warp;
  if (p >= A.n) return;
  const int64_t n = A.n;
  const int n1 = A.n1, ne = A.ne, win = A.win, nodes = n1 * n1 * n1;
  double xp[3];
  int ea[3];
  for (int a = 0; a < 3; ++a) {
    xp[a] = A.x[a * n + p];
    ea[a] = cell_of(xp[a], ne);
  }
  // window factors (exact cutoff decision of the definition)
  for (int u = lane; u < 3 * win; u += 32) {
    const int a = u / win, w = u % win;
    const int o = w / n1 - A.rho, i = w % n1;
    const int ge = wrapi(ea[a] + o, ne);
    const double X = ((double)ge + 0.5 * (A.eta[i] + 1.0)) * A.h;
    const double d = minimg(X - xp[a]);
    kf[warp][a][w] = fabs(d) <= A.rc ? exp(-d * d * A.inv2s2) : 0.0;
    dd[warp][a][w] = d;
  }
  __syncwarp();
  double Z[3], mu[3];
  int lo[3], cnt[3];
  for (int a = 0; a < 3; ++a) {
    double z = 0.0, z1 = 0.0;
    int l = -1, hgh = -2;
    for (int w = 0; w < win; ++w) {
      const double k = kf[warp][a][w];
      if (k != 0.0) {
        if (l < 0) l = w;
        hgh = w;
      }
      z += A.w[w % n1] * k;
      z1 += A.w[w % n1] * k * dd[warp][a][w];
    }
    Z[a] = z;
    mu[a] = z > 0.0 ? z1 / z : 0.0;
    lo[a] = l < 0 ? 0 : l;
    cnt[a] = hgh >= l ? hgh - l + 1 : 0;
  }
  const double q0 = A.q[p], q1 = A.q[n + p], q2 = A.q[2 * n + p], q3 = A.q[3 * n + p];
  double aq[4] = {0, 0, 0, 0}, ax[3] = {0, 0, 0};
  const int nbox = cnt[0] * cnt[1] * cnt[2];
  for (int u = lane; u < nbox; u += 32) {
    const int wx = lo[0] + u % cnt[0];
    const int wy = lo[1] + (u / cnt[0]) % cnt[1];
    const int wz = lo[2] + u / (cnt[0] * cnt[1]);
    const double kx = kf[warp][0][wx], ky = kf[warp][1][wy], kz = kf[warp][2][wz];
    if (kx == 0.0 || ky == 0.0 || kz == 0.0) continue;
    const int gex = wrapi(ea[0] + wx / n1 - A.rho, ne), gey = wrapi(ea[1] + wy / n1 - A.rho, ne),
              gez = wrapi(ea[2] + wz / n1 - A.rho, ne);
    const int64_t e = ((int64_t)gez * ne + gey) * ne + gex;
    const int64_t g = e * 4 * nodes + ((int64_t)(wz % n1) * n1 + (wy % n1)) * n1 + (wx % n1);
    const double G0 = A.G[g], G1 = A.G[g + nodes], G2 = A.G[g + 2 * nodes], G3 = A.G[g + 3 * nodes];
    const double kh = (kx * ky) * kz;
    aq[0] += G0 * kh;
    aq[1] += G1 * kh;
    aq[2] += G2 * kh;
    aq[3] += G3 * kh;
    const double ag = ((G0 * q0 + G1 * q1) + G2 * q2) + G3 * q3;
    const double akh = ag * kh;
    ax[0] += akh * (dd[warp][0][wx] - mu[0]);
    ax[1] += akh * (dd[warp][1][wy] - mu[1]);
    ax[2] += akh * (dd[warp][2][wz] - mu[2]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    for (int c = 0; c < 4; ++c) aq[c] += __shfl_xor_sync(0xffffffffu, aq[c], o);
    for (int a = 0; a < 3; ++a) ax[a] += __shfl_xor_sync(0xffffffffu, ax[a], o);
  }
  if (lane == 0) {
    const double zz = Z[0] * Z[1] * Z[2];
    const double f = zz > 0.0 ? A.scale / zz : 0.0;
    for (int c = 0; c < 4; ++c) A.gq[c * n + p] = aq[c] * f;
    for (int a = 0; a < 3; ++a) A.gx[a * n + p] = ax[a] * f * A.inv_s2;
  }
}

}  // namespace

extern "C" {

pc_status pc_pairs_to_partner(pc_ctx* ctx, int32_t* partner, int64_t n_ids) {
  if (!ctx || !partner || n_ids < 0) return PC_EINVAL;
  cudaError_t e = cudaMemsetAsync(partner, 0xFF, sizeof(int32_t) * (size_t)n_ids, ctx->stream);
  if (e == cudaSuccess && ctx->cfg.n_max > 0) {
    const int64_t cap = ctx->cfg.n_max / 2 + 1;
    k_pairs_to_partner<<<pc_blocks(cap, 256), 256, 0, ctx->stream>>>(n_ids, ctx->counters, ctx->pair_lo,
                                                                      ctx->pair_hi, partner);
    ctx->launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_pairs_to_partner: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}

pc_status pc_collide_replay(pc_ctx* ctx, const pc_particles* in, pc_particles* out, const int32_t* partner,
                            double dt) {
  if (!ctx) return PC_EINVAL;
  if (!in || !out || in->n < 0 || in->n > ctx->cfg.n_max || out->n != in->n ||
      (in->n > 0 && (!partner || !in->x || !in->v || !in->r || !in->m || !out->x || !out->v)) ||
      !(dt > 0.0 && dt < INFINITY)) {
    snprintf(ctx->err, sizeof(ctx->err), "pc_collide_replay: bad arguments");
    return PC_EINVAL;
  }
  if (in->n > 0 && (in->x == out->x || in->v == out->v)) {
    snprintf(ctx->err, sizeof(ctx->err), "pc_collide_replay: in and out must be distinct buffers");
    return PC_EINVAL;
  }
  const int64_t n = in->n;
  if (n == 0) return PC_OK;
  ReplayArgs A;
  A.n = n;
  A.dt = dt;
  A.e = ctx->cfg.restitution;
  A.x = in->x;
  A.v = in->v;
  A.r = in->r;
  A.m = in->m;
  A.q = in->q;
  A.id = in->id;
  A.partner = partner;
  A.xo = out->x;
  A.vo = out->v;
  A.ro = (out->r && out->r != in->r) ? out->r : nullptr;
  A.mo = (out->m && out->m != in->m) ? out->m : nullptr;
  A.ido = (out->id && in->id && out->id != in->id) ? out->id : nullptr;
  A.qo = (out->q && in->q && out->q != in->q) ? out->q : nullptr;
  A.counters = ctx->counters;
  k_replay<<<pc_blocks(n, 256), 256, 0, ctx->stream>>>(A);
  ctx->launches += 1;
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_collide_replay: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}

pc_status pc_collide_adjoint(pc_ctx* ctx, const pc_particles* in, const int32_t* partner, double dt,
                             const double* gx_out, const double* gv_out, double* gx_in, double* gv_in) {
  if (!ctx) return PC_EINVAL;
  if (!in || in->n < 0 || in->n > ctx->cfg.n_max ||
      (in->n > 0 && (!partner || !in->x || !in->v || !in->r || !in->m || !gx_out || !gv_out || !gx_in || !gv_in)) ||
      !(dt > 0.0 && dt < INFINITY)) {
    snprintf(ctx->err, sizeof(ctx->err), "pc_collide_adjoint: bad arguments");
    return PC_EINVAL;
  }
  const int64_t n = in->n;
  if (n == 0) return PC_OK;
  AdjArgs A;
  A.n = n;
  A.dt = dt;
  A.e = ctx->cfg.restitution;
  A.x = in->x;
  A.v = in->v;
  A.r = in->r;
  A.m = in->m;
  A.partner = partner;
  A.gxo = gx_out;
  A.gvo = gv_out;
  A.gxi = gx_in;
  A.gvi = gv_in;
  A.counters = ctx->counters;
  k_collide_adjoint<<<pc_blocks(n, 256), 256, 0, ctx->stream>>>(A);
  ctx->launches += 1;
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_collide_adjoint: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}

pc_status pc_project_adjoint(pc_ctx* ctx, const pc_particles* p, const double* G, double* gq, double* gx) {
  if (!ctx) return PC_EINVAL;
  if (!p || p->n < 0 || p->n > ctx->cfg.n_max || (p->n > 0 && (!p->x || !p->q || !G || !gq || !gx))) {
    snprintf(ctx->err, sizeof(ctx->err), "pc_project_adjoint: bad arguments");
    return PC_EINVAL;
  }
  const int64_t n = p->n;
  if (n == 0) return PC_OK;
  ProjAdjArgs A;
  A.n = n;
  A.ne = ctx->cfg.ne;
  A.n1 = ctx->n1;
  A.rho = ctx->rho;
  A.win = ctx->win;
  A.h = ctx->h;
  A.rc = ctx->cfg.cutoff_sigmas * ctx->cfg.sigma;
  A.inv2s2 = 1.0 / (2.0 * ctx->cfg.sigma * ctx->cfg.sigma);
  A.inv_s2 = 1.0 / (ctx->cfg.sigma * ctx->cfg.sigma);
  const double s2h = 2.0 / ctx->h;
  A.scale = s2h * s2h * s2h;
  for (int i = 0; i < 16; ++i) {
    A.eta[i] = i < ctx->n1 ? ctx->eta[i] : 0.0;
    A.w[i] = i < ctx->n1 ? ctx->w[i] : 0.0;
  }
  A.x = p->x;
  A.q = p->q;
  A.G = G;
  A.gq = gq;
  A.gx = gx;
  k_project_adjoint<<<(unsigned)((n + 3) / 4), 128, 0, ctx->stream>>>(A);
  ctx->launches += 1;
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
  snprintf(ctx->err, sizeof(ctx->err), "pc_project_adjoint: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}

}  // extern "C"
