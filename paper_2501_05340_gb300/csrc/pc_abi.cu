// C ABI of the pc library: context creation, argument validation, scratch
// allocation and the host-side getters. Kernels live in bin.cu, collide.cu and
// project.cu.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pc_internal.cuh"

// Legendre-Gauss rule with n1 points on [-1, 1] (the DGSEM solution points,
// Sec. 3.1): Newton iteration on P_n1 evaluated by Bonnet's recurrence, started
// from the Chebyshev-like estimate cos(pi (k - 1/4) / (n1 + 1/2)).
void pc_gauss_rule(int n1, double* x, double* w) {
  const double pi = 3.141592653589793238462643383279502884;
  for (int k = 1; k <= n1; ++k) {
    double z = cos(pi * (k - 0.25) / (n1 + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 64; ++it) {
      double pm = 1.0, p = z;  // P_0, P_1
      for (int l = 2; l <= n1; ++l) {
        const double pn = ((2 * l - 1) * z * p - (l - 1) * pm) / l;
        pm = p;
        p = pn;
      }
      if (n1 == 1) {
        p = z;
        pm = 1.0;
      }
      dp = n1 * (z * p - pm) / (z * z - 1.0);
      const double step = p / dp;
      z -= step;
      if (fabs(step) <= 1e-16 * fabs(z) + 1e-300) break;
    }
    // final derivative at the converged root
    double pm = 1.0, p = z;
    for (int l = 2; l <= n1; ++l) {
      const double pn = ((2 * l - 1) * z * p - (l - 1) * pm) / l;
      pm = p;
      p = pn;
    }
    dp = n1 * (z * p - pm) / (z * z - 1.0);
    x[n1 - k] = z;  // ascending
    w[n1 - k] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  if (n1 & 1) x[n1 / 2] = 0.0;
}

// exp2(j/64) and ln(2)/64 split into floats for the df32 exponential.
void pc_build_exp_table(DfExpTable* tab) {
  DfExpTable& T = *tab;
  for (int j = 0; j < 64; ++j) {
    const double v = exp2((double)j / 64.0);
    T.th[j] = (float)v;
    T.tl[j] = (float)(v - (double)T.th[j]);
  }
  const double L = log(2.0) / 64.0;
  int ex = 0;
  const double m = frexp(L, &ex);                          // L = m 2^ex, m in [0.5, 1)
  const double L1 = ldexp(floor(ldexp(m, 11)), ex - 11);  // 11 significant bits
  T.L1 = (float)L1;
  T.L2 = (float)(L - L1);
  T.L3 = (float)((L - L1) - (double)T.L2);
  T.inv = (float)(64.0 / log(2.0));
}

namespace {

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

pc_status fail(pc_ctx* ctx, pc_status s, const char* msg) {
  if (ctx) snprintf(ctx->err, sizeof(ctx->err), "%s", msg);
  return s;
}

void free_all(pc_ctx* c) {
  void* ptrs[] = {c->cnt, c->start, c->blocksums, c->key, c->slot, c->perm, c->sx, c->sv, c->sr,
                  c->sid, c->sxf, c->svf, c->srf, c->cand_j, c->cand_t, c->ncand, c->best, c->partner,
                  c->work, c->tcoll, c->pair_lo, c->pair_hi, c->pair_t, c->counters, c->fac, c->sq, c->scell, c->corner, c->reach, c->fxmax, c->trig};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_counters) cudaFreeHost(c->h_counters);
  if (c->ev) {
    for (int i = 0; i < 2 * PC_EVPOOL; ++i) cudaEventDestroy(c->ev[i]);
    free(c->ev);
  }
}

bool particles_ok(const pc_particles* p, int64_t n_max) {
  return p && p->n >= 0 && p->n <= n_max && (p->n == 0 || (p->id && p->x && p->v && p->r && p->m));
}

}  // namespace

extern "C" {

pc_status pc_init(pc_ctx** out, const pc_config* cfg) {
  if (!out) return PC_EINVAL;
  *out = nullptr;
  if (!cfg) return PC_EINVAL;
  const pc_config& c = *cfg;
  if (!(c.n_max > 0 && c.n_max < (int64_t)1 << 31)) return PC_EINVAL;
  if (c.ne < 3 || c.ne > 1024 || c.degree < 0 || c.degree > 15) return PC_EINVAL;
  if (!(c.sigma > 0.0) || !(c.cutoff_sigmas > 0.0) || !(c.restitution >= 0.0 && c.restitution <= 1.0))
    return PC_EINVAL;
  if (c.cutoff_kind != 0 && c.cutoff_kind != 1) return PC_EINVAL;
  // the periodic minimum image names one partner image only while the reach stays
  // below half the box; the search kernels check the actual reach of each step too
  if (!(c.reach_hint > 0.0 && c.reach_hint < 0.5) || c.cand_cap < 0 || c.cand_cap > 32) return PC_EINVAL;
  if (!(c.amp >= 0.0 && c.amp < 0.04)) return PC_EINVAL;
  const double rc = c.cutoff_sigmas * c.sigma;
  // the sphere cutoff serves the curved mesh: in logical space the physical ball of
  // radius rc lies within rc / (1 - L) per axis, L = 2 pi sqrt(3) amp
  const double lip = 6.283185307179586 * 1.7320508075688772 * c.amp;
  const int rho = c.cutoff_kind == 0 ? (int)ceil(rc * c.ne * (1.0 + 1e-12))
                                     : (int)ceil(rc / (1.0 - lip) * c.ne * (1.001) + 1e-9);
  if (rho < 1 || rho > 2 || 2 * rho + 1 > c.ne || !(rc < 0.5)) return PC_EINVAL;
  if ((2 * rho + 1) * (c.degree + 1) > 64) return PC_EINVAL;

  pc_ctx* ctx = (pc_ctx*)calloc(1, sizeof(pc_ctx));
  if (!ctx) return PC_ENOMEM;
  ctx->cfg = c;
  ctx->stream = (cudaStream_t)c.stream;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    free(ctx);
    return PC_ECUDA;
  }
  int64_t nc = (int64_t)floor(1.0 / (c.reach_hint * (1.0 + 1e-9)));
  if (nc < 3) nc = 3;
  if (nc > 1024) nc = 1024;
  while (nc > 3 && nc * nc * nc > ((int64_t)1 << 28)) --nc;
  ctx->nc = (int)nc;
  ctx->ncell = nc * nc * nc;
  ctx->n1 = c.degree + 1;
  ctx->rho = rho;
  ctx->win = (2 * rho + 1) * ctx->n1;
  ctx->h = 1.0 / c.ne;
  ctx->cap = c.cand_cap == 0 ? 16 : c.cand_cap;
  pc_gauss_rule(ctx->n1, ctx->eta, ctx->w);
  pc_build_exp_table(&ctx->exp_tab);

  const int64_t n = c.n_max;
  const int64_t nel = (int64_t)c.ne * c.ne * c.ne;
  ctx->nbins_max = std::max<int64_t>(ctx->ncell, nel);
  const int64_t nb1 = ctx->nbins_max + 1;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  chk(dalloc(&ctx->cnt, nb1));
  chk(dalloc(&ctx->start, nb1));
  chk(dalloc(&ctx->blocksums, nb1 / PC_SCAN_TILE + 2));
  chk(dalloc(&ctx->key, n));
  chk(dalloc(&ctx->slot, n));
  chk(dalloc(&ctx->perm, n));
  chk(dalloc(&ctx->sx, 3 * n));
  chk(dalloc(&ctx->sv, 3 * n));
  chk(dalloc(&ctx->sr, n));
  chk(dalloc(&ctx->sid, n));
  chk(dalloc(&ctx->sxf, 3 * n));
  chk(dalloc(&ctx->svf, 3 * n));
  chk(dalloc(&ctx->srf, n));
  chk(dalloc(&ctx->cand_j, (int64_t)ctx->cap * n));
  chk(dalloc(&ctx->cand_t, (int64_t)ctx->cap * n));
  chk(dalloc(&ctx->ncand, n));
  chk(dalloc(&ctx->best, n));
  chk(dalloc(&ctx->partner, n));
  chk(dalloc(&ctx->work, n));
  chk(dalloc(&ctx->scell, n));
  chk(dalloc(&ctx->tcoll, n));
  chk(dalloc(&ctx->pair_lo, n / 2 + 1));
  chk(dalloc(&ctx->pair_hi, n / 2 + 1));
  chk(dalloc(&ctx->pair_t, n / 2 + 1));
  chk(dalloc(&ctx->counters, CNT_N));
  ctx->rs = (3 * ctx->win + 4 + 1) & ~1;
  chk(dalloc(&ctx->fac, (int64_t)ctx->rs * n));
  chk(dalloc(&ctx->sq, 4 * n));
  chk(dalloc(&ctx->reach, n));
  chk(dalloc(&ctx->fxmax, 8));
  chk(dalloc(&ctx->corner, 36 * nel));
  chk(dalloc(&ctx->trig, (int64_t)(c.ne + 2 * rho) * ctx->n1));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_counters, sizeof(unsigned long long) * CNT_N);
  if (e == cudaSuccess) e = cudaMemset(ctx->counters, 0, sizeof(unsigned long long) * CNT_N);
  if (e != cudaSuccess) {
    pc_status s = (e == cudaErrorMemoryAllocation) ? PC_ENOMEM : PC_ECUDA;
    free_all(ctx);
    free(ctx);
    cudaGetLastError();
    return s;
  }
  snprintf(ctx->err, sizeof(ctx->err), "no error");
  *out = ctx;
  return PC_OK;
}

pc_status pc_collide(pc_ctx* ctx, const pc_particles* in, pc_particles* out, double dt) {
  if (!ctx) return PC_EINVAL;
  if (!particles_ok(in, ctx->cfg.n_max) || !particles_ok(out, ctx->cfg.n_max) || in->n != out->n)
    return fail(ctx, PC_EINVAL, "pc_collide: bad particle arrays");
  if (in->n > 0 && (in->x == out->x || in->v == out->v || in->id == out->id || in->r == out->r || in->m == out->m))
    return fail(ctx, PC_EINVAL, "pc_collide: in and out must be distinct buffers");
  if (in->n > 0 && in->q && (!out->q || out->q == in->q))
    return fail(ctx, PC_EINVAL, "pc_collide: out->q must be a distinct buffer when in->q is given");
  if (!(dt > 0.0 && dt < INFINITY)) return fail(ctx, PC_EINVAL, "pc_collide: dt must be positive and finite");
  return pc_collide_impl(ctx, in, out, dt);
}

pc_status pc_collide_rot(pc_ctx* ctx, const pc_particles* in, pc_particles* out, const double* w_in, double* w_out,
                         double mu, double dt) {
  if (!ctx) return PC_EINVAL;
  if (!particles_ok(in, ctx->cfg.n_max) || !particles_ok(out, ctx->cfg.n_max) || in->n != out->n)
    return fail(ctx, PC_EINVAL, "pc_collide_rot: bad particle arrays");
  if (in->n > 0 && (in->x == out->x || in->v == out->v || in->id == out->id || in->r == out->r || in->m == out->m))
    return fail(ctx, PC_EINVAL, "pc_collide_rot: in and out must be distinct buffers");
  if (in->n > 0 && in->q && (!out->q || out->q == in->q))
    return fail(ctx, PC_EINVAL, "pc_collide_rot: out->q must be a distinct buffer when in->q is given");
  if (in->n > 0 && (!w_in || !w_out || w_in == w_out))
    return fail(ctx, PC_EINVAL, "pc_collide_rot: w_in and w_out must be distinct non-NULL buffers");
  if (!(mu >= 0.0 && mu < INFINITY)) return fail(ctx, PC_EINVAL, "pc_collide_rot: mu must be finite and >= 0");
  if (!(dt > 0.0 && dt < INFINITY)) return fail(ctx, PC_EINVAL, "pc_collide_rot: dt must be positive and finite");
  return pc_collide_impl(ctx, in, out, dt, w_in, w_out, mu);
}

pc_status pc_project(pc_ctx* ctx, const pc_particles* p, double* field) {
  if (!ctx) return PC_EINVAL;
  if (ctx->cfg.cutoff_kind != 0) return fail(ctx, PC_EINVAL, "pc_project: needs the box cutoff (cutoff_kind 0)");
  if (!particles_ok(p, ctx->cfg.n_max) || !field || (p->n > 0 && !p->q))
    return fail(ctx, PC_EINVAL, "pc_project: bad arguments");
  return pc_project_impl(ctx, p, field);
}

pc_status pc_eval_field(pc_ctx* ctx, const pc_particles* p, const double* field, int32_t nvar, double* out) {
  if (!ctx) return PC_EINVAL;
  if (!particles_ok(p, ctx->cfg.n_max) || nvar < 1 || nvar > 16 || (p->n > 0 && (!field || !out)))
    return fail(ctx, PC_EINVAL, "pc_eval_field: bad arguments");
  return pc_eval_field_impl(ctx, p, field, nvar, out);
}

pc_status pc_drag_sources(pc_ctx* ctx, const pc_particles* p, const double* fluid, double mu_f, double* q) {
  if (!ctx) return PC_EINVAL;
  if (!particles_ok(p, ctx->cfg.n_max) || (p->n > 0 && (!fluid || !q)))
    return fail(ctx, PC_EINVAL, "pc_drag_sources: bad arguments");
  if (!(mu_f > 0.0 && mu_f < INFINITY)) return fail(ctx, PC_EINVAL, "pc_drag_sources: mu_f must be positive");
  return pc_drag_sources_impl(ctx, p, fluid, mu_f, q);
}

pc_status pc_project_idw(pc_ctx* ctx, const pc_particles* p, double* field) {
  if (!ctx) return PC_EINVAL;
  if (!particles_ok(p, ctx->cfg.n_max) || !field || (p->n > 0 && !p->q))
    return fail(ctx, PC_EINVAL, "pc_project_idw: bad arguments");
  return pc_project_idw_impl(ctx, p, field);
}

pc_status pc_project_dirac(pc_ctx* ctx, const pc_particles* p, double* field) {
  if (!ctx) return PC_EINVAL;
  if (!particles_ok(p, ctx->cfg.n_max) || !field || (p->n > 0 && !p->q))
    return fail(ctx, PC_EINVAL, "pc_project_dirac: bad arguments");
  return pc_project_dirac_impl(ctx, p, field);
}

pc_status pc_set_pair_policy(pc_ctx* ctx, int32_t policy) {
  if (!ctx) return PC_EINVAL;
  if (policy != PC_PAIRS_EARLIEST && policy != PC_PAIRS_SFC_FIRST)
    return fail(ctx, PC_EINVAL, "pc_set_pair_policy: unknown policy");
  ctx->pair_policy = policy;
  return PC_OK;
}

int32_t pc_cells_per_side(const pc_ctx* ctx) { return ctx ? ctx->nc : 0; }

static bool particles_f32_ok(const pc_particles_f32* p, int64_t n_max) {
  return p && p->n >= 0 && p->n <= n_max && (p->n == 0 || (p->id && p->cell && p->o && p->v && p->r && p->m));
}

pc_status pc_quantize(pc_ctx* ctx, const pc_particles* in, pc_particles_f32* out) {
  if (!ctx) return PC_EINVAL;
  if (!particles_ok(in, ctx->cfg.n_max) || !particles_f32_ok(out, ctx->cfg.n_max) || in->n != out->n)
    return fail(ctx, PC_EINVAL, "pc_quantize: bad particle arrays");
  return pc_quantize_impl(ctx, in, out);
}

pc_status pc_collide_f32(pc_ctx* ctx, const pc_particles_f32* in, pc_particles_f32* out, double dt) {
  if (!ctx) return PC_EINVAL;
  if (!particles_f32_ok(in, ctx->cfg.n_max) || !particles_f32_ok(out, ctx->cfg.n_max) || in->n != out->n)
    return fail(ctx, PC_EINVAL, "pc_collide_f32: bad particle arrays");
  if (in->n > 0 && (in->cell == out->cell || in->o == out->o || in->v == out->v || in->id == out->id ||
                    in->r == out->r || in->m == out->m))
    return fail(ctx, PC_EINVAL, "pc_collide_f32: in and out must be distinct buffers");
  if (in->n > 0 && in->q && (!out->q || out->q == in->q))
    return fail(ctx, PC_EINVAL, "pc_collide_f32: out->q must be a distinct buffer when in->q is given");
  if (!(dt > 0.0 && dt < INFINITY)) return fail(ctx, PC_EINVAL, "pc_collide_f32: dt must be positive and finite");
  return pc_collide_f32_impl(ctx, in, out, dt);
}

pc_status pc_project_f32(pc_ctx* ctx, const pc_particles_f32* p, float* field, int32_t tc_type) {
  if (!ctx) return PC_EINVAL;
  if (!particles_f32_ok(p, ctx->cfg.n_max) || !field || (p->n > 0 && !p->q) ||
      (tc_type != PC_TC_F16 && tc_type != PC_TC_BF16))
    return fail(ctx, PC_EINVAL, "pc_project_f32: bad arguments");
  if (ctx->n1 > 8 || ctx->win > 32)
    return fail(ctx, PC_EINVAL, "pc_project_f32: needs N + 1 <= 8 and (2 rho + 1)(N + 1) <= 32");
  if (ctx->cfg.cutoff_kind != 0) return fail(ctx, PC_EINVAL, "pc_project_f32: needs the box cutoff");
  return pc_project_f32_impl(ctx, p, field, tc_type);
}

pc_status pc_collide_replay_f32(pc_ctx* ctx, const pc_particles_f32* in, pc_particles_f32* out, const int32_t* partner,
                                double dt) {
  if (!ctx) return PC_EINVAL;
  if (!particles_f32_ok(in, ctx->cfg.n_max) || !particles_f32_ok(out, ctx->cfg.n_max) || in->n != out->n ||
      (in->n > 0 && !partner))
    return fail(ctx, PC_EINVAL, "pc_collide_replay_f32: bad arguments");
  if (in->n > 0 && (in->cell == out->cell || in->o == out->o || in->v == out->v))
    return fail(ctx, PC_EINVAL, "pc_collide_replay_f32: in and out cell, o, v must be distinct buffers");
  if (!(dt > 0.0 && dt < INFINITY))
    return fail(ctx, PC_EINVAL, "pc_collide_replay_f32: dt must be positive and finite");
  return pc_collide_replay_f32_impl(ctx, in, out, partner, dt);
}

pc_status pc_collide_adjoint_f32(pc_ctx* ctx, const pc_particles_f32* in, const int32_t* partner, double dt,
                                 const float* gx_out, const float* gv_out, float* gx_in, float* gv_in) {
  if (!ctx) return PC_EINVAL;
  if (!particles_f32_ok(in, ctx->cfg.n_max) ||
      (in->n > 0 && (!partner || !gx_out || !gv_out || !gx_in || !gv_in)))
    return fail(ctx, PC_EINVAL, "pc_collide_adjoint_f32: bad arguments");
  if (in->n > 0 && (gx_in == gx_out || gv_in == gv_out || gx_in == gv_out || gv_in == gx_out))
    return fail(ctx, PC_EINVAL, "pc_collide_adjoint_f32: input and output cotangents must be distinct buffers");
  if (!(dt > 0.0 && dt < INFINITY))
    return fail(ctx, PC_EINVAL, "pc_collide_adjoint_f32: dt must be positive and finite");
  return pc_collide_adjoint_f32_impl(ctx, in, partner, dt, gx_out, gv_out, gx_in, gv_in);
}

pc_status pc_project_adjoint_f32(pc_ctx* ctx, const pc_particles_f32* p, const float* G, float* gq, float* gx) {
  if (!ctx) return PC_EINVAL;
  if (!particles_f32_ok(p, ctx->cfg.n_max) || (p->n > 0 && (!p->q || !G || !gq || !gx)))
    return fail(ctx, PC_EINVAL, "pc_project_adjoint_f32: bad arguments");
  if (ctx->cfg.cutoff_kind != 0) return fail(ctx, PC_EINVAL, "pc_project_adjoint_f32: needs the box cutoff");
  return pc_project_adjoint_f32_impl(ctx, p, G, gq, gx);
}

pc_status pc_project_curved_f32(pc_ctx* ctx, const pc_particles_f32* p, float* field) {
  if (!ctx) return PC_EINVAL;
  if (!particles_f32_ok(p, ctx->cfg.n_max) || !field || (p->n > 0 && !p->q))
    return fail(ctx, PC_EINVAL, "pc_project_curved_f32: bad arguments");
  if (ctx->cfg.cutoff_kind != 1)
    return fail(ctx, PC_EINVAL, "pc_project_curved_f32: needs the sphere cutoff (cutoff_kind 1)");
  if (ctx->n1 * ctx->n1 * ctx->n1 > 1024)
    return fail(ctx, PC_EINVAL, "pc_project_curved_f32: needs (N + 1)^3 <= 1024");
  return pc_project_curved_f32_impl(ctx, p, field);
}

pc_status pc_sync(pc_ctx* ctx) {
  if (!ctx) return PC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    snprintf(ctx->err, sizeof(ctx->err), "CUDA: %s", cudaGetErrorString(e));
    return PC_ECUDA;
  }
  unsigned long long st = 0;
  e = cudaMemcpy(&st, ctx->counters + CNT_STATUS, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return PC_ECUDA;
  if (st) {
    // indexed by pc_status; PC_ENOMEM and PC_ECUDA are host-side codes and never raised on the GPU
    static const char* names[] = {"ok",
                                  "invalid particle data (position outside [0,1), radius, mass or velocity)",
                                  "out of memory",
                                  "CUDA error",
                                  "matching did not converge",
                                  "candidate list overflow: raise cand_cap",
                                  "a bounded wait in a kernel expired",
                                  "a given pair has no contact within the step (replay / adjoint)"};
    const unsigned long long nnames = sizeof(names) / sizeof(names[0]);
    snprintf(ctx->err, sizeof(ctx->err), "device: %s", st < nnames ? names[st] : "unknown");
    const unsigned long long z = 0;
    cudaMemcpy(ctx->counters + CNT_STATUS, &z, sizeof(z), cudaMemcpyHostToDevice);
  }
  return (pc_status)st;
}

pc_status pc_get_stats(pc_ctx* ctx, pc_stats* out) {
  if (!ctx || !out) return PC_EINVAL;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess ||
      cudaMemcpy(ctx->h_counters, ctx->counters, sizeof(unsigned long long) * CNT_N, cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return fail(ctx, PC_ECUDA, "pc_get_stats: CUDA error");
  const unsigned long long* h = ctx->h_counters;
  out->pairs = (int64_t)h[CNT_PAIRS];
  out->candidates = (int64_t)h[CNT_CANDS];
  out->worklist = (int64_t)h[CNT_WORK];
  out->rounds = (int64_t)h[CNT_ROUNDS];
  out->fp64_solves = (int64_t)h[CNT_SOLVES];
  out->max_candidates = (int64_t)h[CNT_MAXCAND];
  out->cells_per_side = ctx->nc;
  out->stencil = (int32_t)h[CNT_STENCIL];
  out->device_status = (int32_t)h[CNT_STATUS];
  out->kernel_launches = ctx->launches;
  return (pc_status)h[CNT_STATUS];
}

pc_status pc_get_pairs(pc_ctx* ctx, int32_t* ids, double* t, int64_t cap, int64_t* npairs) {
  if (!ctx || !npairs || cap < 0 || (cap > 0 && (!ids || !t))) return PC_EINVAL;
  unsigned long long np = 0;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess ||
      cudaMemcpy(&np, ctx->counters + CNT_PAIRS, sizeof(np), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(ctx, PC_ECUDA, "pc_get_pairs: CUDA error");
  if (np > (unsigned long long)(ctx->cfg.n_max / 2 + 1))
    return fail(ctx, PC_ECAPACITY, "pc_get_pairs: pair count exceeds the pair buffers");
  std::vector<int32_t> lo(np), hi(np);
  std::vector<double> tt(np);
  if (np && (cudaMemcpy(lo.data(), ctx->pair_lo, 4 * np, cudaMemcpyDeviceToHost) != cudaSuccess ||
             cudaMemcpy(hi.data(), ctx->pair_hi, 4 * np, cudaMemcpyDeviceToHost) != cudaSuccess ||
             cudaMemcpy(tt.data(), ctx->pair_t, 8 * np, cudaMemcpyDeviceToHost) != cudaSuccess))
    return fail(ctx, PC_ECUDA, "pc_get_pairs: CUDA error");
  std::vector<int64_t> order(np);
  for (uint64_t a = 0; a < np; ++a) order[a] = (int64_t)a;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return lo[a] < lo[b]; });
  const int64_t m = std::min<int64_t>(cap, (int64_t)np);
  for (int64_t a = 0; a < m; ++a) {
    ids[2 * a] = lo[order[a]];
    ids[2 * a + 1] = hi[order[a]];
    t[a] = tt[order[a]];
  }
  *npairs = (int64_t)np;
  return PC_OK;
}

pc_status pc_set_timing(pc_ctx* ctx, int on) {
  if (!ctx) return PC_EINVAL;
  if (on && !ctx->ev) {
    ctx->ev = (cudaEvent_t*)calloc(2 * PC_EVPOOL, sizeof(cudaEvent_t));
    if (!ctx->ev) return fail(ctx, PC_ENOMEM, "pc_set_timing: out of host memory");
    for (int i = 0; i < 2 * PC_EVPOOL; ++i)
      if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess) {
        for (int k = 0; k < i; ++k) cudaEventDestroy(ctx->ev[k]);
        free(ctx->ev);
        ctx->ev = nullptr;
        return fail(ctx, PC_ECUDA, "pc_set_timing: cudaEventCreate failed");
      }
  }
  ctx->timing = on ? 1 : 0;
  return PC_OK;
}

pc_status pc_get_timing(pc_ctx* ctx, double* ms, int64_t* count) {
  if (!ctx) return PC_EINVAL;
  if (ms)
    for (int p = 0; p < PC_NPHASE; ++p) ms[p] = 0.0;
  if (count)
    for (int p = 0; p < PC_NPHASE; ++p) count[p] = 0;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return fail(ctx, PC_ECUDA, "pc_get_timing: CUDA error");
  for (int i = 0; i < ctx->nrec; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ctx->ev[2 * i], ctx->ev[2 * i + 1]) != cudaSuccess)
      return fail(ctx, PC_ECUDA, "pc_get_timing: cudaEventElapsedTime failed");
    const int p = ctx->rec_phase[i];
    if (ms) ms[p] += t;
    if (count) count[p] += 1;
  }
  ctx->nrec = 0;
  return PC_OK;
}

const char* pc_last_error(const pc_ctx* ctx) { return ctx ? ctx->err : "null context"; }

void pc_destroy(pc_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  free(ctx);
}

}  // extern "C"
