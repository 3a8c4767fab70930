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

struct FactorArgs {
  int64_t n;
  int ne, n1, rho, win;
  double h, rc, inv2s2;
  double eta[16], w[16];  // Legendre-Gauss nodes and weights on [-1, 1]
  const int32_t* perm;
  const double* x;
  const double* q;
  double* fac;  // [3][win][n]
  double* sq;   // [4][n]
};

// fac[a][w][k] = k_a(X_w - x_a) / Za for the window node w = (o + rho) n1 + i of
// element (own element + o), with k_a(d) = exp(-d^2 / (2 sigma^2)) for |d| <= rc
// and 0 beyond; Za = sum_w w_i k_a.
__global__ void k_proj_factors(FactorArgs F) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = F.n;
  if (k >= n) return;
  const int64_t p = F.perm[k];
  for (int a = 0; a < 3; ++a) {
    const double xa = F.x[a * n + p];
    const int ea = cell_of(xa, F.ne);
    double Z = 0.0;
    for (int w = 0; w < F.win; ++w) {
      const int o = w / F.n1 - F.rho, i = w % F.n1;
      const int ge = wrapi(ea + o, F.ne);
      const double X = ((double)ge + 0.5 * (F.eta[i] + 1.0)) * F.h;
      const double d = minimg(X - xa);
      const double f = fabs(d) <= F.rc ? exp(-d * d * F.inv2s2) : 0.0;
      F.fac[((int64_t)a * F.win + w) * n + k] = f;
      Z += F.w[i] * f;
    }
    const double iz = 1.0 / Z;
    for (int w = 0; w < F.win; ++w) F.fac[((int64_t)a * F.win + w) * n + k] *= iz;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) F.sq[c * n + k] = F.q[c * n + p];
}

struct GatherArgs {
  int64_t n;
  int ne, n1, rho, win, nwarps;
  double scale;  // (2/h)^3
  const int32_t* start;
  const double* fac;
  const double* sq;
  double* field;
};

__global__ void k_proj_gather(GatherArgs G) {
  extern __shared__ double smem[];
  const int n1 = G.n1, nodes = n1 * n1 * n1, NW = G.nwarps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* acc = smem;                               // [NW][4][nodes]
  double* stage = smem + (size_t)NW * 4 * nodes;    // [NW][3*16 + 4]
  double* my = acc + (size_t)warp * 4 * nodes;
  double* fs = stage + warp * 52;
  for (int a = threadIdx.x; a < NW * 4 * nodes; a += blockDim.x) acc[a] = 0.0;
  __syncthreads();
  const int64_t n = G.n;
  const int ne = G.ne;
  const int e = blockIdx.x;
  const int ex = e % ne, ey = (e / ne) % ne, ez = e / (ne * ne);
  int turn = 0;  // running particle count over the neighbour ranges, split round-robin over warps
  for (int dz = -G.rho; dz <= G.rho; ++dz)
    for (int dy = -G.rho; dy <= G.rho; ++dy)
      for (int dx = -G.rho; dx <= G.rho; ++dx) {
        const int nb = (wrapi(ez + dz, ne) * ne + wrapi(ey + dy, ne)) * ne + wrapi(ex + dx, ne);
        const int beg = G.start[nb], end = G.start[nb + 1];
        // this element sits at offset -d in the window of a particle of element e + d
        const int wx = (G.rho - dx) * n1, wy = (G.rho - dy) * n1, wz = (G.rho - dz) * n1;
        for (int j = beg; j < end; ++j, ++turn) {
          if (turn % NW != warp) continue;
          for (int u = lane; u < 3 * n1; u += 32) {
            const int a = u / n1, i = u % n1;
            const int wa = a == 0 ? wx : (a == 1 ? wy : wz);
            fs[a * 16 + i] = G.fac[((int64_t)a * G.win + wa + i) * n + j];
          }
          if (lane < 4) fs[48 + lane] = G.sq[(int64_t)lane * n + j];
          __syncwarp();
          int lo[3], cntv[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            int l = n1, h = -1;
            for (int i = 0; i < n1; ++i)
              if (fs[a * 16 + i] != 0.0) {
                l = min(l, i);
                h = i;
              }
            lo[a] = l;
            cntv[a] = h - l + 1;
          }
          if (cntv[0] > 0 && cntv[1] > 0 && cntv[2] > 0) {
            const int nbox = cntv[0] * cntv[1] * cntv[2];
            const double q0 = fs[48], q1 = fs[49], q2 = fs[50], q3 = fs[51];
            for (int u = lane; u < nbox; u += 32) {
              const int i = lo[0] + u % cntv[0];
              const int jj = lo[1] + (u / cntv[0]) % cntv[1];
              const int kk = lo[2] + u / (cntv[0] * cntv[1]);
              const double wgt = (fs[i] * fs[16 + jj]) * fs[32 + kk];
              const int g = (kk * n1 + jj) * n1 + i;
              my[g] += q0 * wgt;
              my[nodes + g] += q1 * wgt;
              my[2 * nodes + g] += q2 * wgt;
              my[3 * nodes + g] += q3 * wgt;
            }
          }
          __syncwarp();
        }
      }
  __syncthreads();
  double* out = G.field + (int64_t)e * 4 * nodes;
  for (int a = threadIdx.x; a < 4 * nodes; a += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += acc[(size_t)w * 4 * nodes + a];
    out[a] = s * G.scale;
  }
}

}  // namespace

static int gather_warps(int n1, size_t* smem) {
  const size_t nodes = (size_t)n1 * n1 * n1;
  const size_t per = (4 * nodes + 52) * sizeof(double);
  int nw = (int)((200 * 1024) / per);
  if (nw > 8) nw = 8;
  if (nw < 1) nw = 1;
  *smem = per * nw;
  return nw;
}

pc_status pc_project_impl(pc_ctx* ctx, const pc_particles* p, double* field) {
  const int64_t n = p->n;
  cudaStream_t st = ctx->stream;
  const int ne = ctx->cfg.ne;
  const int64_t nel = (int64_t)ne * ne * ne;
  cudaError_t e = cudaMemsetAsync(ctx->cnt, 0, sizeof(int32_t) * (size_t)nel, st);
  if (e != cudaSuccess) goto fail;
  {
    const int tb = pc_phase_begin(ctx, PC_PH_PBIN);
    if (n > 0) {
      k_elem_keys<<<pc_blocks(n, 256), 256, 0, st>>>(n, p->x, ne, ctx->key, ctx->slot, ctx->cnt, ctx->counters);
      ctx->launches += 1;
    }
    e = pc_bin_finish(n, nel, ctx->key, ctx->slot, p->id, ctx->cnt, ctx->start, ctx->blocksums, ctx->perm, st,
                      &ctx->launches);
    pc_phase_end(ctx, tb);
  }
  if (e != cudaSuccess) goto fail;
  if (n > 0) {
    FactorArgs F;
    F.n = n;
    F.ne = ne;
    F.n1 = ctx->n1;
    F.rho = ctx->rho;
    F.win = ctx->win;
    F.h = ctx->h;
    F.rc = ctx->cfg.cutoff_sigmas * ctx->cfg.sigma;
    F.inv2s2 = 1.0 / (2.0 * ctx->cfg.sigma * ctx->cfg.sigma);
    for (int i = 0; i < 16; ++i) {
      F.eta[i] = i < ctx->n1 ? ctx->eta[i] : 0.0;
      F.w[i] = i < ctx->n1 ? ctx->w[i] : 0.0;
    }
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
    GatherArgs G;
    G.n = n;
    G.ne = ne;
    G.n1 = ctx->n1;
    G.rho = ctx->rho;
    G.win = ctx->win;
    size_t smem = 0;
    G.nwarps = gather_warps(ctx->n1, &smem);
    const double s = 2.0 / ctx->h;
    G.scale = s * s * s;
    G.start = ctx->start;
    G.fac = ctx->fac;
    G.sq = ctx->sq;
    G.field = field;
    e = cudaFuncSetAttribute(k_proj_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) goto fail;
    const int td = pc_phase_begin(ctx, PC_PH_DEPOSIT);
    k_proj_gather<<<(unsigned)nel, 32 * G.nwarps, smem, st>>>(G);
    ctx->launches += 1;
    pc_phase_end(ctx, td);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
fail:
  snprintf(ctx->err, sizeof(ctx->err), "pc_project: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}
