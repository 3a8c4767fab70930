// Projection on the curved periodic mesh (arXiv 2501.05340 deposition, Sec. 2.3 /
// 4.2, with a non-separable Gaussian shape function in physical space):
//   x = Phi(xi) = xi + amp (sin 2pi xi_y sin 2pi xi_z, sin 2pi xi_z sin 2pi xi_x, sin 2pi xi_x sin 2pi xi_y),
//   field[g][c] = sum_p q[c][p] K(X_g - x_p) / Z_p, Z_p = sum_g W_g K(X_g - x_p),
//   W_g = w_i w_j w_k (h/2)^3 det DPhi(xi_g), K(d) = exp(-|d|^2/(2 sigma^2)) for |d| <= rc.
// Steps: Newton's method on Phi(xi) = x locates every particle in logical space
// (the localisation of Sec. 3.2) and bins it by logical element; per particle Z_p
// over the logical box that bounds the physical ball of radius rc (|Phi(a) - Phi(b)|
// >= (1 - L)|a - b| with L = 2 pi sqrt(3) amp); per element a gather over the
// particles of the 2 rho + 1 logical neighbours, culled by the element's bounding
// box. FP32 factors and accumulation; positions as double-float so that node to
// particle distances keep their precision; cutoff decisions within 2e-4 relative
// of the cutoff are made in FP64 with the plain definition. Compiled with -fmad=false.
#include <math.h>
#include <string.h>

#include "df32.cuh"
#include "pc_internal.cuh"

namespace {

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

__device__ __forceinline__ float minimgf(float d) {
  if (d > 0.5f) return d - 1.0f;
  if (d < -0.5f) return d + 1.0f;
  return d;
}

__device__ __forceinline__ double minimg(double d) {
  if (d > 0.5) return d - 1.0;
  if (d < -0.5) return d + 1.0;
  return d;
}

// 2^x for the kernel's arguments (-7 < x <= 0 inside the cutoff): the hardware
// approximation, the same in the normalisation and in the deposit.
__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void raise_status(unsigned long long* counters, int code) {
  atomicMax(&counters[CNT_STATUS], (unsigned long long)code);
}

// Position (c + o)/nc of a cell-relative coordinate as double-float.
__device__ __forceinline__ f2 pos_df(int c, float o, f2 inv_nc) { return df_mul(two_sum((float)c, o), inv_nc); }

struct LocArgs {
  int64_t n;
  int nc, ne;
  float amp;
  f2 inv_nc;
  const int32_t* cell;
  const float* o;
  float* xi;  // [3][n], input order
  int32_t *key, *slot, *cnt;
  unsigned long long* counters;
};

// Newton's method on Phi(xi) = x (residual taken in the periodic minimum image),
// 8 iterations from xi = x; the map's perturbation has Lipschitz constant < 0.5,
// so the iteration contracts quadratically.
__global__ void k_curved_locate(LocArgs A) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  if (p >= n) return;
  const int32_t cl = A.cell[p];
  const int nc = A.nc;
  if (!(cl >= 0 && (int64_t)cl < (int64_t)nc * nc * nc)) raise_status(A.counters, PC_EINVAL);
  const int32_t cs = cl < 0 ? 0 : cl;
  const int c3[3] = {cs % nc, (cs / nc) % nc, cs / (nc * nc)};
  float x[3], xi[3];
  for (int a = 0; a < 3; ++a) {
    const float oa = A.o[a * n + p];
    if (!(oa >= 0.0f && oa < 1.0f)) raise_status(A.counters, PC_EINVAL);
    const f2 xd = pos_df(c3[a], oa, A.inv_nc);
    x[a] = xd.h;
    xi[a] = xd.h;
  }
  const float g = 6.283185307179586f * A.amp;
  for (int it = 0; it < 8; ++it) {
    float s[3], c[3];
    for (int a = 0; a < 3; ++a) sincospif(2.0f * xi[a], &s[a], &c[a]);
    const float F0 = minimgf(xi[0] + A.amp * s[1] * s[2] - x[0]);
    const float F1 = minimgf(xi[1] + A.amp * s[2] * s[0] - x[1]);
    const float F2 = minimgf(xi[2] + A.amp * s[0] * s[1] - x[2]);
    // J = I + g [[0, c1 s2, s1 c2], [c0 s2, 0, s0 c2], [c0 s1, s0 c1, 0]]
    const float a01 = g * c[1] * s[2], a02 = g * s[1] * c[2];
    const float a10 = g * c[0] * s[2], a12 = g * s[0] * c[2];
    const float a20 = g * c[0] * s[1], a21 = g * s[0] * c[1];
    const float det = 1.0f * (1.0f - a12 * a21) - a01 * (a10 - a12 * a20) + a02 * (a10 * a21 - a20);
    const float d0 = (F0 * (1.0f - a12 * a21) - a01 * (F1 - a12 * F2) + a02 * (F1 * a21 - F2)) / det;
    const float d1 = ((F1 - a12 * F2) - F0 * (a10 - a12 * a20) + a02 * (a10 * F2 - a20 * F1)) / det;
    const float d2 = ((F2 - a21 * F1) - a01 * (a10 * F2 - a20 * F1) + F0 * (a10 * a21 - a20)) / det;
    xi[0] -= d0;
    xi[1] -= d1;
    xi[2] -= d2;
  }
  int e[3];
  for (int a = 0; a < 3; ++a) {
    float w = xi[a] - floorf(xi[a]);
    if (w >= 1.0f) w = 0.0f;
    xi[a] = w;
    int ea = (int)(w * (float)A.ne);
    e[a] = ea < 0 ? 0 : (ea >= A.ne ? A.ne - 1 : ea);
    A.xi[a * n + p] = w;
  }
  const int k = (e[2] * A.ne + e[1]) * A.ne + e[0];
  A.key[p] = k;
  A.slot[p] = atomicAdd(&A.cnt[k], 1);
}

// sin and cos of 2 pi X at the Gauss coordinates X = (e + s_i) h of one axis (the map
// is the same on every axis), from the double-float coordinate; rho elements of
// periodic images on either side, so that window nodes index it without wrapping.
struct TrigArgs {
  int ne, n1, rho;
  f2 h;
  float s[16];
  float2* trig;  // [(ne + 2 rho) n1]: entry t holds global node index t - rho n1, wrapped
};

__global__ void k_curved_trig(TrigArgs T) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (T.ne + 2 * T.rho) * T.n1) return;
  const int e = wrapi(t / T.n1 - T.rho, T.ne);
  const f2 xg = df_mul(two_sum((float)e, T.s[t % T.n1]), T.h);
  float sn, cs;
  sincospif(2.0f * xg.h, &sn, &cs);
  T.trig[t] = make_float2(sn, cs);
}

struct CPrepArgs {
  int64_t n;
  int nc, ne, n1, rho, win;
  float amp, rcl, rc2f, c2l, inv_h;
  f2 inv_nc, h;
  double hd, rc;
  float s[16], wq[16];
  double eta[16];
  float S[64];  // window coordinates: S[w] = (w / n1 + s[w % n1]) h
  const float2* trig;  // per-axis table, entry g + rho n1 for global node index g
  const int32_t* perm;
  const int32_t* cell;
  const float* o;
  const float* xi;
  const float* q;
  float4* rec;  // [n][3]: (x0h x0l x1h x1l) (x2h x2l 1/Z q0) (q1 q2 q3 -)
};

// Inside-cutoff decision for a node: float distance squared r2 against rc^2, and the
// plain FP64 definition within 2e-4 relative of the edge (x_p = (c + o)/nc).
__device__ __forceinline__ bool inside_cut(float r2, float rc2f, const int c3[3], const float o3[3], int nc,
                                           const double xig[3], float amp, double rc) {
  if (r2 < rc2f * 0.9998f) return true;
  if (r2 > rc2f * 1.0002f) return false;
  const double tp = 6.283185307179586476925286766559;
  double s[3];
  for (int a = 0; a < 3; ++a) s[a] = sin(tp * xig[a]);
  const double X[3] = {xig[0] + (double)amp * s[1] * s[2], xig[1] + (double)amp * s[2] * s[0],
                       xig[2] + (double)amp * s[0] * s[1]};
  double d[3];
  for (int a = 0; a < 3; ++a) d[a] = minimg(X[a] - ((double)c3[a] + (double)o3[a]) / (double)nc);
  const double d2s = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
  return d2s <= rc * rc;
}

// First window node at or after window coordinate v, less one (clamped to [0, win]):
// a conservative start of the nodes within reach of v.
__device__ __forceinline__ int win_from(float v, float inv_h, const float* s, int n1, int win) {
  const float u = v * inv_h;
  const int eo = (int)floorf(u);
  if (eo < 0) return 0;
  if (eo * n1 >= win) return win;
  const float t = u - (float)eo;
  int i = 0;
  while (i < n1 && s[i] < t) ++i;
  const int w = eo * n1 + i - 1;
  return w < 0 ? 0 : (w > win ? win : w);
}

// Last window node at or before v, plus one, as an exclusive end (clamped to [0, win]).
__device__ __forceinline__ int win_to(float v, float inv_h, const float* s, int n1, int win) {
  const float u = v * inv_h;
  const int eo = (int)floorf(u);
  if (eo < 0) return 0;
  if (eo * n1 >= win) return win;
  const float t = u - (float)eo;
  int i = 0;
  while (i < n1 && s[i] <= t) ++i;
  const int w = eo * n1 + i + 1;
  return w > win ? win : w;
}

// Z_p over the nodes of the physical ball, particle per thread (sorted order). The
// window of (2 rho + 1) n1 nodes per axis around the particle's logical element is
// walked plane by plane, row by row and node by node over the index ranges that the
// logical ball of radius rcl can reach (|Phi(a) - Phi(b)| >= (1 - L)|a - b|; the
// ranges are widened by a node on each side and every node is decided by its
// physical distance). Node to particle offsets: the window offset of the node from
// the particle's logical position, plus the particle's logical-minus-physical offset
// delta, plus the map's perturbation at the node; sines and cosines come from the
// per-axis table.
__global__ void __launch_bounds__(128) k_curved_prep(CPrepArgs A) {
  // window coordinates and weights in shared memory: lanes index them at different
  // nodes, which kernel-parameter reads would serialise
  __shared__ float S[64], WQ[64];
  if (threadIdx.x < 64) {
    S[threadIdx.x] = A.S[threadIdx.x];
    WQ[threadIdx.x] = A.wq[threadIdx.x % A.n1];
  }
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  if (k >= n) return;
  const int64_t p = A.perm[k];
  const int nc = A.nc, ne = A.ne, n1 = A.n1, rho = A.rho, win = A.win;
  const int32_t cl = A.cell[p] < 0 ? 0 : A.cell[p];
  const int c3[3] = {cl % nc, (cl / nc) % nc, cl / (nc * nc)};
  float o3[3], cw[3], dl[3];
  f2 x[3];
  int g0[3];
  for (int a = 0; a < 3; ++a) {
    o3[a] = A.o[a * n + p];
    x[a] = pos_df(c3[a], o3[a], A.inv_nc);
    const float xia = A.xi[a * n + p];
    int e = (int)(xia * (float)ne);
    e = e < 0 ? 0 : (e >= ne ? ne - 1 : e);
    // the particle in window coordinates: xi - (e - rho) h, and delta = xi - x
    const f2 base = df_mul(two_sum((float)(e - rho), 0.0f), A.h);
    cw[a] = (xia - base.h) - base.l;
    dl[a] = minimgf(xia - x[a].h) - x[a].l;
    g0[a] = e * n1;  // table entry of window node 0: global node index (e - rho) n1, plus rho n1
  }
  const float amp = A.amp, g = 6.283185307179586f * amp, rcl = A.rcl, rcl2 = rcl * rcl;
  const float cut_hi = A.rc2f * 1.0002f;
  float Z = 0.0f;
  const int z0 = win_from(cw[2] - rcl, A.inv_h, A.s, n1, win), z1 = win_to(cw[2] + rcl, A.inv_h, A.s, n1, win);
  for (int wz = z0; wz < z1; ++wz) {
    const float lz = S[wz] - cw[2];
    const float ry2 = rcl2 - lz * lz;
    if (ry2 < 0.0f) continue;
    const int gz = g0[2] + wz;
    const float2 tz = A.trig[gz];
    const float dz0 = lz + dl[2];
    const float ry = sqrtf(ry2);
    const int y0 = win_from(cw[1] - ry, A.inv_h, A.s, n1, win), y1 = win_to(cw[1] + ry, A.inv_h, A.s, n1, win);
    for (int wy = y0; wy < y1; ++wy) {
      const float ly = S[wy] - cw[1];
      const float rx2 = ry2 - ly * ly;
      if (rx2 < 0.0f) continue;
      const int gy = g0[1] + wy;
      const float2 ty = A.trig[gy];
      const float dy0 = ly + dl[1];
      const float rx = sqrtf(rx2);
      // row constants: perturbations and Jacobian entries that do not involve x
      const float pxr = amp * ty.x * tz.x;
      const float az = amp * tz.x, ay = amp * ty.x;
      const float a01 = g * ty.y * tz.x, a02 = g * ty.x * tz.y;
      const float gsz = g * tz.x, gcz = g * tz.y, gsy = g * ty.x, gcy = g * ty.y;
      const float wyz = WQ[wy] * WQ[wz];
      const int x0 = win_from(cw[0] - rx, A.inv_h, A.s, n1, win), x1 = win_to(cw[0] + rx, A.inv_h, A.s, n1, win);
      for (int wx = x0; wx < x1; ++wx) {
        const float lx = S[wx] - cw[0];
        const int gx = g0[0] + wx;
        const float2 tx = A.trig[gx];
        // this unit is compiled without implicit contraction (double-float helpers); the
        // FP32 arithmetic of the node pairs places its multiply-adds explicitly
        const float dx = (lx + dl[0]) + pxr;
        const float dy = fmaf(az, tx.x, dy0);
        const float dz = fmaf(ay, tx.x, dz0);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (r2 > cut_hi) continue;
        if (r2 >= A.rc2f * 0.9998f) {
          const int gg[3] = {gx, gy, gz};
          double xig[3];
          for (int a = 0; a < 3; ++a)
            xig[a] = ((double)wrapi(gg[a] / n1 - rho, ne) + 0.5 * (A.eta[gg[a] % n1] + 1.0)) * A.hd;
          if (!inside_cut(r2, A.rc2f, c3, o3, nc, xig, amp, A.rc)) continue;
        }
        const float a10 = gsz * tx.y, a12 = gcz * tx.x;
        const float a20 = gsy * tx.y, a21 = gcy * tx.x;
        const float det = fmaf(a02, fmaf(a10, a21, -a20), fmaf(-a01, fmaf(-a12, a20, a10), fmaf(-a12, a21, 1.0f)));
        const float W = WQ[wx] * wyz * det;
        Z = fmaf(W, ex2f(-r2 * A.c2l), Z);
      }
    }
  }
  const float hh = 0.5f * A.h.h;
  Z *= hh * hh * hh;
  const float iz = Z > 0.0f ? 1.0f / Z : 0.0f;
  float4* rp = A.rec + 3 * k;
  rp[0] = make_float4(x[0].h, x[0].l, x[1].h, x[1].l);
  rp[1] = make_float4(x[2].h, x[2].l, iz, A.q[p]);
  rp[2] = make_float4(A.q[n + p], A.q[2 * n + p], A.q[3 * n + p], 0.0f);
}

struct CDepArgs {
  int64_t n;
  int nc, ne, n1, rho;
  float amp, rc2f, rcf, c2l;
  f2 h;
  double hd, rc;
  float s[16];
  double eta[16];
  const float2* trig;  // per-axis table, entry g + rho n1 for global node index g
  const int32_t* start;
  const int32_t* perm;  // for the FP64 edge decisions (stored cell + offset)
  const int32_t* cell;
  const float* o;
  const float4* rec;
  float* field;
};

// One CTA per element, one thread per node. Node positions relative to the element's
// logical corner E: (s_i h) + the map's perturbation. The particles of the
// neighbouring logical elements are staged in batches (one per thread) as their
// positions relative to E (double-float difference, minimum image) with a bounding-box
// test; every node then adds q_c K / Z of the staged particles that pass.
__global__ void __launch_bounds__(64, 12) k_curved_deposit(CDepArgs A) {
  extern __shared__ float4 sm4[];
  const int nodes = blockDim.x;  // n1^3
  float4* st = sm4;                                      // [nodes][2]: (relative x, 1/Z), q
  int* keep = (int*)(sm4 + 2 * nodes);                   // [nodes]: staged particle index + 1, or 0
  int* clist = keep + nodes;                             // [nodes]: compacted positions of the kept ones
  __shared__ float bbox[6];
  __shared__ int pre[126], rbeg[126];
  __shared__ int wcnt[32];
  __shared__ float red[6][32];
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5, nwarps = (nodes + 31) / 32;
  const int n1 = A.n1, ne = A.ne, rho = A.rho, span = 2 * rho + 1, nrange = span * span * span;
  const int e = blockIdx.x;
  const int ex = e % ne, ey = (e / ne) % ne, ez = e / (ne * ne);
  const int i = t % n1, j = (t / n1) % n1, k = t / (n1 * n1);
  const int el[3] = {ex, ey, ez}, li[3] = {i, j, k};
  float sn[3];
  f2 E[3];
  for (int a = 0; a < 3; ++a) {
    sn[a] = A.trig[(el[a] + rho) * n1 + li[a]].x;
    E[a] = df_mul(two_sum((float)el[a], 0.0f), A.h);
  }
  const float amp = A.amp;
  const float X[3] = {A.s[i] * A.h.h + amp * sn[1] * sn[2], A.s[j] * A.h.h + amp * sn[2] * sn[0],
                      A.s[k] * A.h.h + amp * sn[0] * sn[1]};
  // bounding box of the element's relative node positions
  {
    const unsigned wmask = nodes - 32 * wp >= 32 ? 0xffffffffu : ((1u << (nodes - 32 * wp)) - 1u);
    float lo[3] = {X[0], X[1], X[2]}, hi[3] = {X[0], X[1], X[2]};
    for (int o = 16; o > 0; o >>= 1)
      for (int a = 0; a < 3; ++a) {
        const int src = lane + o;
        const float l2 = __shfl_down_sync(wmask, lo[a], o), h2 = __shfl_down_sync(wmask, hi[a], o);
        if (src < 32 && ((wmask >> src) & 1u)) {
          lo[a] = fminf(lo[a], l2);
          hi[a] = fmaxf(hi[a], h2);
        }
      }
    if (lane == 0)
      for (int a = 0; a < 3; ++a) {
        red[a][wp] = lo[a];
        red[3 + a][wp] = hi[a];
      }
  }
  // neighbour ranges and their prefix sum (first warp)
  if (wp == 0) {
    int total = 0;
    for (int r0 = 0; r0 < nrange; r0 += 32) {
      const int r = r0 + lane;
      int cnt = 0;
      if (r < nrange) {
        const int dx = r % span - rho, dy = (r / span) % span - rho, dz = r / (span * span) - rho;
        const int nb = (wrapi(ez + dz, ne) * ne + wrapi(ey + dy, ne)) * ne + wrapi(ex + dx, ne);
        const int b0 = A.start[nb];
        cnt = A.start[nb + 1] - b0;
        rbeg[r] = b0;
      }
      const unsigned m = __ballot_sync(0xffffffffu, r < nrange);
      int x = cnt;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (r < nrange) pre[r + 1] = total + x;
      total += __shfl_sync(0xffffffffu, x, 31);
      (void)m;
    }
    if (lane == 0) pre[0] = 0;
  }
  __syncthreads();
  if (t == 0)
    for (int a = 0; a < 3; ++a) {
      float lo = red[a][0], hi = red[3 + a][0];
      for (int w2 = 1; w2 < nwarps; ++w2) {
        lo = fminf(lo, red[a][w2]);
        hi = fmaxf(hi, red[3 + a][w2]);
      }
      bbox[a] = lo;
      bbox[3 + a] = hi;
    }
  __syncthreads();
  const float cen[3] = {0.5f * (bbox[0] + bbox[3]), 0.5f * (bbox[1] + bbox[4]), 0.5f * (bbox[2] + bbox[5])};
  const float hw[3] = {0.5f * (bbox[3] - bbox[0]), 0.5f * (bbox[4] - bbox[1]), 0.5f * (bbox[5] - bbox[2])};
  const float cut = A.rcf * 1.0002f + 1e-6f;
  const float cut_hi = A.rc2f * 1.0002f, cut_lo = A.rc2f * 0.9998f;
  const int total = pre[nrange];
  int top = 1;
  while (2 * top <= nrange) top *= 2;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int base = 0; base < total; base += nodes) {
    const int idx = base + t;
    int kp = 0;
    if (idx < total) {
      int r = 0;
      for (int stp = top; stp > 0; stp >>= 1)
        if (r + stp < nrange && pre[r + stp] <= idx) r += stp;
      const int jj = rbeg[r] + (idx - pre[r]);
      const float4 r0 = A.rec[3 * (int64_t)jj], r1 = A.rec[3 * (int64_t)jj + 1], r2 = A.rec[3 * (int64_t)jj + 2];
      const f2 xp[3] = {{r0.x, r0.y}, {r0.z, r0.w}, {r1.x, r1.y}};
      float rel[3];
      float d2 = 0.0f;
      for (int a = 0; a < 3; ++a) {
        const f2 dd = df_add(xp[a], df_neg(E[a]));
        rel[a] = minimgf(dd.h + dd.l);
        const float ex_ = fmaxf(fabsf(rel[a] - cen[a]) - hw[a], 0.0f);
        d2 += ex_ * ex_;
      }
      st[2 * t] = make_float4(rel[0], rel[1], rel[2], r1.z);
      st[2 * t + 1] = make_float4(r1.w, r2.x, r2.y, r2.z);
      kp = d2 <= cut * cut ? jj + 1 : 0;
    }
    keep[t] = kp;
    // compact the staged particles that pass the box test (order kept); the mask holds
    // the lanes this warp has (n1^3 need not be a multiple of 32)
    const int wl = nodes - 32 * wp;
    const unsigned wmask = wl >= 32 ? 0xffffffffu : ((1u << wl) - 1u);
    const unsigned bal = __ballot_sync(wmask, kp != 0);
    if (lane == 0) wcnt[wp] = __popc(bal);
    __syncthreads();
    int woff = 0, nkept = 0;
    for (int w2 = 0; w2 < nwarps; ++w2) {
      if (w2 < wp) woff += wcnt[w2];
      nkept += wcnt[w2];
    }
    if (kp) clist[woff + __popc(bal & ((1u << lane) - 1u))] = t;
    __syncthreads();
    for (int u = 0; u < nkept; ++u) {
      const int q = clist[u];
      const float4 s0 = st[2 * q];
      const float d0 = X[0] - s0.x, d1 = X[1] - s0.y, d2 = X[2] - s0.z;
      // explicit multiply-adds: the unit is compiled without implicit contraction
      const float r2s = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
      if (r2s > cut_hi) continue;
      if (r2s >= cut_lo) {
        const int64_t pj = A.perm[keep[q] - 1];
        const int32_t cl = A.cell[pj] < 0 ? 0 : A.cell[pj];
        const int nc = A.nc;
        const int c3[3] = {cl % nc, (cl / nc) % nc, cl / (nc * nc)};
        const float o3[3] = {A.o[pj], A.o[A.n + pj], A.o[2 * A.n + pj]};
        double xig[3];
        for (int a = 0; a < 3; ++a) xig[a] = ((double)el[a] + 0.5 * (A.eta[li[a]] + 1.0)) * A.hd;
        if (!inside_cut(r2s, A.rc2f, c3, o3, nc, xig, amp, A.rc)) continue;
      }
      const float4 s1 = st[2 * q + 1];
      const float K = ex2f(-r2s * A.c2l) * s0.w;
      acc[0] = fmaf(s1.x, K, acc[0]);
      acc[1] = fmaf(s1.y, K, acc[1]);
      acc[2] = fmaf(s1.z, K, acc[2]);
      acc[3] = fmaf(s1.w, K, acc[3]);
    }
    __syncthreads();
  }
  float* out = A.field + (int64_t)e * 4 * nodes;
  for (int c = 0; c < 4; ++c) out[c * nodes + t] = acc[c];
}

}  // namespace

pc_status pc_project_curved_f32_impl(pc_ctx* ctx, const pc_particles_f32* p, float* field) {
  const int64_t n = p->n;
  cudaStream_t st = ctx->stream;
  const int ne = ctx->cfg.ne;
  const int64_t nel = (int64_t)ne * ne * ne;
  const double inv = 1.0 / (double)ctx->nc;
  const f2 inv_nc = {(float)inv, (float)(inv - (double)(float)inv)};
  const f2 hdf = {(float)ctx->h, (float)(ctx->h - (double)(float)ctx->h)};
  const double rc = ctx->cfg.cutoff_sigmas * ctx->cfg.sigma;
  float sgl[16];
  for (int i = 0; i < ctx->n1; ++i) sgl[i] = (float)(0.5 * (ctx->eta[i] + 1.0));
  cudaError_t e = cudaMemsetAsync(ctx->cnt, 0, sizeof(int32_t) * (size_t)nel, st);
  if (e != cudaSuccess) goto fail;
  {
    const int tb = pc_phase_begin(ctx, PC_PH_PBIN);
    {
      // the per-axis sine and cosine table at the Gauss coordinates
      TrigArgs T;
      memset(&T, 0, sizeof(T));
      T.ne = ne;
      T.n1 = ctx->n1;
      T.rho = ctx->rho;
      T.h = hdf;
      memcpy(T.s, sgl, sizeof(sgl));
      T.trig = ctx->trig;
      const int nt = (ne + 2 * ctx->rho) * ctx->n1;
      k_curved_trig<<<(nt + 127) / 128, 128, 0, st>>>(T);
      ctx->launches += 1;
    }
    if (n > 0) {
      LocArgs L;
      L.n = n;
      L.nc = ctx->nc;
      L.ne = ne;
      L.amp = (float)ctx->cfg.amp;
      L.inv_nc = inv_nc;
      L.cell = p->cell;
      L.o = p->o;
      L.xi = ctx->sxf;
      L.key = ctx->key;
      L.slot = ctx->slot;
      L.cnt = ctx->cnt;
      L.counters = ctx->counters;
      k_curved_locate<<<pc_blocks(n, 256), 256, 0, st>>>(L);
      ctx->launches += 1;
    }
    e = pc_bin_finish(n, nel, ctx->key, ctx->slot, p->id, ctx->cnt, ctx->start, ctx->blocksums, ctx->perm, st,
                      &ctx->launches);
    pc_phase_end(ctx, tb);
  }
  if (e != cudaSuccess) goto fail;
  if (n > 0) {
    CPrepArgs P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.nc = ctx->nc;
    P.ne = ne;
    P.n1 = ctx->n1;
    P.rho = ctx->rho;
    P.win = ctx->win;
    P.amp = (float)ctx->cfg.amp;
    const double lip = 6.283185307179586 * 1.7320508075688772 * ctx->cfg.amp;
    P.rcl = (float)(rc / (1.0 - lip) * 1.001 + 1e-6);
    P.rc2f = (float)(rc * rc);
    P.c2l = (float)(1.4426950408889634 / (2.0 * ctx->cfg.sigma * ctx->cfg.sigma));
    P.inv_h = (float)ne;
    P.inv_nc = inv_nc;
    P.h = hdf;
    P.hd = ctx->h;
    P.rc = rc;
    for (int i = 0; i < ctx->n1; ++i) {
      P.s[i] = sgl[i];
      P.wq[i] = (float)ctx->w[i];
      P.eta[i] = ctx->eta[i];
    }
    for (int w = 0; w < ctx->win; ++w)
      P.S[w] = (float)(((double)(w / ctx->n1) + 0.5 * (ctx->eta[w % ctx->n1] + 1.0)) * ctx->h);
    P.trig = ctx->trig;
    P.perm = ctx->perm;
    P.cell = p->cell;
    P.o = p->o;
    P.xi = ctx->sxf;
    P.q = p->q;
    P.rec = (float4*)ctx->fac;
    const int tf = pc_phase_begin(ctx, PC_PH_FACTORS);
    k_curved_prep<<<pc_blocks(n, 128), 128, 0, st>>>(P);
    ctx->launches += 1;
    pc_phase_end(ctx, tf);
  }
  {
    CDepArgs D;
    memset(&D, 0, sizeof(D));
    D.n = n;
    D.nc = ctx->nc;
    D.ne = ne;
    D.n1 = ctx->n1;
    D.rho = ctx->rho;
    D.amp = (float)ctx->cfg.amp;
    D.rc2f = (float)(rc * rc);
    D.rcf = (float)rc;
    D.c2l = (float)(1.4426950408889634 / (2.0 * ctx->cfg.sigma * ctx->cfg.sigma));
    D.h = hdf;
    D.hd = ctx->h;
    D.rc = rc;
    for (int i = 0; i < ctx->n1; ++i) {
      D.s[i] = sgl[i];
      D.eta[i] = ctx->eta[i];
    }
    D.trig = ctx->trig;
    D.start = ctx->start;
    D.perm = ctx->perm;
    D.cell = p->cell;
    D.o = p->o;
    D.rec = (const float4*)ctx->fac;
    D.field = field;
    const int nodes = ctx->n1 * ctx->n1 * ctx->n1;
    const size_t smem = (size_t)nodes * (2 * sizeof(float4) + 2 * sizeof(int));
    const int td = pc_phase_begin(ctx, PC_PH_DEPOSIT);
    k_curved_deposit<<<(unsigned)nel, nodes, smem, st>>>(D);
    ctx->launches += 1;
    pc_phase_end(ctx, td);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) return PC_OK;
fail:
  snprintf(ctx->err, sizeof(ctx->err), "pc_project_curved_f32: %s", cudaGetErrorString(e));
  return PC_ECUDA;
}
