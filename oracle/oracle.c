/*
 * CPU oracle for the particle collision and projection operator
 * (arXiv 2501.05340). TEST INFRASTRUCTURE ONLY: tests, the smoke check and the
 * benchmark's CPU baseline load it; the product path never does.
 *
 * Plain FP64 C, compiled with -O2 -ffp-contract=off -fno-fast-math so that
 * every + - * / sqrt below is one IEEE double operation in the written order.
 * Function-by-function citations:
 *   or_gauss_legendre      Sec. 3.1 (Legendre-Gauss points of the DGSEM)
 *   or_contact_time        Sec. 3.3, Eqs. collision-detect 1-2 and the rules after them
 *   or_candidates_*        Sec. 4.3 (halo criterion |d| <= d_max + r + r')
 *   or_match_*             Sec. 4.3 (one collision per particle per step)
 *   or_respond_advance     Sec. 2.4 (J_n = -m_r (1+e) v_r.n, frictionless), Sec. 3.3 update
 *   or_project             Sec. 2.3 / 4.2 (deposition operator P, Gaussian shape function)
 *   or_project_idw/_dirac  Sec. 2.3 / 4.2 (corner-node and nearest-DOF deposition)
 *   or_respond_advance_rot Sec. 2.4 (friction and rotation)
 *   or_eval_field          Sec. 3.2 (field evaluation: the DG solution at the particles)
 *   or_drag_sources        Sec. 2.2 / 2.3 (drag force and its momentum and energy sources)
 * Readings where the paper is silent or garbled are listed at each function.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ Gauss */

/* Legendre polynomial P_n(x) and P_{n-1}(x) by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static void legendre(int n, double x, double* pn, double* pn1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *pn1 = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *pn1 = p0;
}

int or_gauss_legendre(int n1, double* eta, double* w) {
  if (n1 < 1 || n1 > 64 || !eta || !w) return 1;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n1; ++i) {
    /* initial guess near the i-th largest root, then Newton on P_n */
    double x = cos(pi * (i + 0.75) / (n1 + 0.5));
    double pn = 0, pn1 = 0, dp = 0;
    for (int it = 0; it < 100; ++it) {
      legendre(n1, x, &pn, &pn1);
      dp = n1 * (x * pn - pn1) / (x * x - 1.0);
      double dx = pn / dp;
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    legendre(n1, x, &pn, &pn1);
    dp = n1 * (x * pn - pn1) / (x * x - 1.0);
    eta[n1 - 1 - i] = x; /* ascending order */
    w[n1 - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  if (n1 % 2 == 1) eta[n1 / 2] = 0.0; /* the middle root is exactly zero */
  return 0;
}

/* ------------------------------------------------------------------ contact */

/* Periodic minimum image of a coordinate difference of two points in [0,1). */
static double minimg(double d) {
  if (d > 0.5) return d - 1.0;
  if (d < -0.5) return d + 1.0;
  return d;
}

/* Same in a periodic box of length L (L = 1 gives minimg exactly). */
static double minimg_box(double d, double L) {
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

/* Reading of the garbled Eq. collision-detect 2: dx_p = x_1 - x_2 and
 * dv_p = v_1 - v_2. With a = dv.dv, b = dx.dv, c = dx.dx - R^2 the roots of
 * a t^2 + 2 b t + c = 0 are both positive iff c > 0 and b < 0 (b < 0 also says the
 * pair is closing in), real and distinct iff b^2 - a c > 0 (a grazing
 * double root carries no normal velocity). The smaller root is written as
 * c / (-b + sqrt(b^2 - a c)), the cancellation-free form of (-b - sqrt(.))/a.
 * The root must satisfy t <= dt (inclusive). */
static double contact_time_box(const double xi[3], const double xj[3], const double vi[3], const double vj[3],
                               double R, double dt, double L) {
  double dx0 = minimg_box(xi[0] - xj[0], L);
  double dx1 = minimg_box(xi[1] - xj[1], L);
  double dx2 = minimg_box(xi[2] - xj[2], L);
  double dv0 = vi[0] - vj[0];
  double dv1 = vi[1] - vj[1];
  double dv2 = vi[2] - vj[2];
  double a = (dv0 * dv0 + dv1 * dv1) + dv2 * dv2;
  double b = (dx0 * dv0 + dx1 * dv1) + dx2 * dv2;
  double c = ((dx0 * dx0 + dx1 * dx1) + dx2 * dx2) - R * R;
  if (!(b < 0.0)) return INFINITY;
  if (!(c > 0.0)) return INFINITY;
  double disc = b * b - a * c;
  if (!(disc > 0.0)) return INFINITY;
  double t = c / (-b + sqrt(disc));
  if (t <= dt) return t;
  return INFINITY;
}

double or_contact_time(const double xi[3], const double xj[3], const double vi[3], const double vj[3],
                       double ri, double rj, double dt) {
  return contact_time_box(xi, xj, vi, vj, ri + rj, dt, 1.0);
}

static void load3(const double* a, int64_t n, int64_t i, double out[3]) {
  out[0] = a[i];
  out[1] = a[n + i];
  out[2] = a[2 * n + i];
}

int64_t or_candidates_bruteforce(int64_t n, const double* x, const double* v, const double* r, double dt,
                                 int64_t cap, int64_t* ci, int64_t* cj, double* ct) {
  int64_t cnt = 0;
  for (int64_t i = 0; i < n; ++i) {
    double xi[3], vi[3];
    load3(x, n, i, xi);
    load3(v, n, i, vi);
    for (int64_t j = i + 1; j < n; ++j) {
      double xj[3], vj[3];
      load3(x, n, j, xj);
      load3(v, n, j, vj);
      double t = or_contact_time(xi, xj, vi, vj, r[i], r[j], dt);
      if (t <= dt) {
        if (cnt < cap) { ci[cnt] = i; cj[cnt] = j; ct[cnt] = t; }
        ++cnt;
      }
    }
  }
  return cnt;
}

static int64_t cell_of(double y, int64_t nc) {
  int64_t c = (int64_t)floor(y * (double)nc);
  if (c < 0) c = 0;
  if (c >= nc) c = nc - 1;
  return c;
}

int64_t or_candidates_cells(int64_t n, const double* x, const double* v, const double* r, double dt,
                            int64_t cap, int64_t* ci, int64_t* cj, double* ct) {
  /* Any pair with a root t <= dt starts within R + |dv| dt <= 2 r_max + 2 v_max dt
   * of each other (Sec. 4.3: d_max from the fastest particle and the time step). */
  double rmax = 0.0, v2max = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (r[i] > rmax) rmax = r[i];
    double s = v[i] * v[i] + v[n + i] * v[n + i] + v[2 * n + i] * v[2 * n + i];
    if (s > v2max) v2max = s;
  }
  double reach = (2.0 * rmax + 2.0 * sqrt(v2max) * dt) * (1.0 + 1e-9) + 1e-12;
  int64_t nc = (int64_t)floor(1.0 / reach);
  if (nc > 1024) nc = 1024;
  if (nc < 3) return or_candidates_bruteforce(n, x, v, r, dt, cap, ci, cj, ct);
  int64_t ncell = nc * nc * nc;
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!head || !next || !cell) { free(head); free(next); free(cell); return -1; }
  for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
  for (int64_t i = n - 1; i >= 0; --i) {
    int64_t c = (cell_of(x[2 * n + i], nc) * nc + cell_of(x[n + i], nc)) * nc + cell_of(x[i], nc);
    cell[i] = c;
    next[i] = head[c];
    head[c] = i;
  }
  int64_t cnt = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t cx = cell[i] % nc, cy = (cell[i] / nc) % nc, cz = cell[i] / (nc * nc);
    double xi[3], vi[3];
    load3(x, n, i, xi);
    load3(v, n, i, vi);
    for (int64_t dz = -1; dz <= 1; ++dz)
      for (int64_t dy = -1; dy <= 1; ++dy)
        for (int64_t dx = -1; dx <= 1; ++dx) {
          int64_t c = (((cz + dz + nc) % nc) * nc + (cy + dy + nc) % nc) * nc + (cx + dx + nc) % nc;
          for (int64_t j = head[c]; j >= 0; j = next[j]) {
            if (j <= i) continue;
            double xj[3], vj[3];
            load3(x, n, j, xj);
            load3(v, n, j, vj);
            double t = or_contact_time(xi, xj, vi, vj, r[i], r[j], dt);
            if (t <= dt) {
              if (cnt < cap) { ci[cnt] = i; cj[cnt] = j; ct[cnt] = t; }
              ++cnt;
            }
          }
        }
  }
  free(head);
  free(next);
  free(cell);
  return cnt;
}

/* ------------------------------------------------------------------ matching */

typedef struct {
  double t;
  int32_t lo, hi; /* ids, lo < hi */
  int64_t i, j;   /* indices */
} edge_t;

static int edge_cmp(const void* pa, const void* pb) {
  const edge_t* a = (const edge_t*)pa;
  const edge_t* b = (const edge_t*)pb;
  if (a->t < b->t) return -1;
  if (a->t > b->t) return 1;
  if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
  if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
  return 0;
}

/* Reading: the paper commits the first valid pair found in its deterministic
 * element order and removes both particles from further tests. Here the order
 * is the earliest contact first, ties broken by (smaller id, larger id). */
int64_t or_match_greedy(int64_t n, const int32_t* id, int64_t ncand, const int64_t* ci, const int64_t* cj,
                        const double* ct, int64_t* partner, double* tc) {
  for (int64_t i = 0; i < n; ++i) { partner[i] = -1; tc[i] = INFINITY; }
  edge_t* e = (edge_t*)malloc(sizeof(edge_t) * (size_t)(ncand > 0 ? ncand : 1));
  if (!e) return -1;
  for (int64_t k = 0; k < ncand; ++k) {
    int32_t a = id[ci[k]], b = id[cj[k]];
    e[k].t = ct[k];
    e[k].lo = a < b ? a : b;
    e[k].hi = a < b ? b : a;
    e[k].i = ci[k];
    e[k].j = cj[k];
  }
  qsort(e, (size_t)ncand, sizeof(edge_t), edge_cmp);
  int64_t pairs = 0;
  for (int64_t k = 0; k < ncand; ++k) {
    if (partner[e[k].i] < 0 && partner[e[k].j] < 0) {
      partner[e[k].i] = e[k].j;
      partner[e[k].j] = e[k].i;
      tc[e[k].i] = e[k].t;
      tc[e[k].j] = e[k].t;
      ++pairs;
    }
  }
  free(e);
  return pairs;
}

/* (t, id of other) order seen from one endpoint. */
static int better(double t1, int32_t id1, double t2, int32_t id2) {
  if (t1 < t2) return 1;
  if (t1 > t2) return 0;
  return id1 < id2;
}

int64_t or_match_rounds(int64_t n, const int32_t* id, int64_t ncand, const int64_t* ci, const int64_t* cj,
                        const double* ct, int64_t* partner, double* tc, int64_t* rounds) {
  for (int64_t i = 0; i < n; ++i) { partner[i] = -1; tc[i] = INFINITY; }
  /* adjacency lists (CSR) of the candidate graph */
  int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* adj = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * ncand + 1));
  int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* best = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!deg || !adj || !fill || !best) { free(deg); free(adj); free(fill); free(best); return -1; }
  for (int64_t k = 0; k < ncand; ++k) { deg[ci[k] + 1]++; deg[cj[k] + 1]++; }
  for (int64_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
  for (int64_t k = 0; k < ncand; ++k) {
    adj[deg[ci[k]] + fill[ci[k]]++] = k;
    adj[deg[cj[k]] + fill[cj[k]]++] = k;
  }
  int64_t pairs = 0, nr = 0;
  for (;;) {
    int any = 0;
    for (int64_t i = 0; i < n; ++i) {
      best[i] = -1;
      if (partner[i] >= 0) continue;
      double bt = INFINITY;
      int32_t bid = 0;
      for (int64_t a = deg[i]; a < deg[i + 1]; ++a) {
        int64_t k = adj[a];
        int64_t o = ci[k] == i ? cj[k] : ci[k];
        if (partner[o] >= 0) continue;
        if (best[i] < 0 || better(ct[k], id[o], bt, bid)) { best[i] = o; bt = ct[k]; bid = id[o]; }
      }
      if (best[i] >= 0) any = 1;
    }
    if (!any) break;
    int64_t committed = 0;
    for (int64_t i = 0; i < n; ++i) {
      int64_t j = best[i];
      if (j > i && best[j] == i) {
        partner[i] = j;
        partner[j] = i;
        /* the edge's contact time */
        for (int64_t a = deg[i]; a < deg[i + 1]; ++a) {
          int64_t k = adj[a];
          if ((ci[k] == i && cj[k] == j) || (ci[k] == j && cj[k] == i)) { tc[i] = tc[j] = ct[k]; break; }
        }
        ++committed;
      }
    }
    ++nr;
    pairs += committed;
    if (committed == 0) break; /* cannot happen for a strict total order; guards the loop */
  }
  if (rounds) *rounds = nr;
  free(deg);
  free(adj);
  free(fill);
  free(best);
  return pairs;
}

/* ------------------------------------------------------------------ response */

/* y - floor(y) lies in [0,1]; a tiny negative y rounds it to exactly 1.0, which
 * is mapped back to 0.0 so that every coordinate stays in [0,1). */
static double wrap01(double y) {
  double w = y - floor(y);
  if (w == 1.0) w = 0.0;
  return w;
}

/* Frictionless hard-sphere response. With s = dx + t dv the contact vector
 * (from particle j to particle i, dx = minimg(x_i - x_j), dv = v_i - v_j),
 * n = -s/|s| is the unit normal from i to j (Sec. 2.4 points the normal from the
 * first sphere of the pair to the second). v_r = v_i - v_j, m_r = m_i m_j/(m_i + m_j),
 * J = -m_r (1 + e) (v_r . n), v_i' = v_i + (J/m_i) n, v_j' = v_j - (J/m_j) n.
 * Reading of the garbled position update of Sec. 3.3: the particle moves with
 * its old velocity to the contact point and with its new one for the rest of
 * the step, x' = x + t v + (dt - t) v'. Free particles: x' = x + dt v. */
void or_respond_advance(int64_t n, double* x, double* v, const double* m, const int64_t* partner,
                        const double* tc, double e, double dt) {
  double* xn = (double*)malloc(sizeof(double) * (size_t)(3 * n > 0 ? 3 * n : 1));
  double* vn = (double*)malloc(sizeof(double) * (size_t)(3 * n > 0 ? 3 * n : 1));
  if (!xn || !vn) { free(xn); free(vn); return; }
  for (int64_t i = 0; i < n; ++i) {
    int64_t j = partner[i];
    if (j < 0) {
      for (int k = 0; k < 3; ++k) {
        vn[k * n + i] = v[k * n + i];
        xn[k * n + i] = x[k * n + i] + dt * v[k * n + i];
      }
      continue;
    }
    double t = tc[i];
    double dx[3], dv[3], s[3], nrm[3];
    for (int k = 0; k < 3; ++k) {
      dx[k] = minimg(x[k * n + i] - x[k * n + j]);
      dv[k] = v[k * n + i] - v[k * n + j];
    }
    for (int k = 0; k < 3; ++k) s[k] = dx[k] + t * dv[k];
    double sl = sqrt((s[0] * s[0] + s[1] * s[1]) + s[2] * s[2]);
    for (int k = 0; k < 3; ++k) nrm[k] = -s[k] / sl;
    double vrn = (dv[0] * nrm[0] + dv[1] * nrm[1]) + dv[2] * nrm[2];
    double mr = (m[i] * m[j]) / (m[i] + m[j]);
    double J = -mr * (1.0 + e) * vrn;
    double gi = J / m[i];
    for (int k = 0; k < 3; ++k) {
      double vold = v[k * n + i];
      double vnew = vold + gi * nrm[k];
      vn[k * n + i] = vnew;
      xn[k * n + i] = (x[k * n + i] + t * vold) + (dt - t) * vnew;
    }
  }
  for (int64_t a = 0; a < 3 * n; ++a) {
    v[a] = vn[a];
    x[a] = wrap01(xn[a]);
  }
  free(xn);
  free(vn);
}

/* Response with Coulomb friction and rotation (Sec. 2.4: the jump relations of
 * linear and angular momentum, J = J_n n + J_t t, J_n = -m_r (1+e) v_r.n, the
 * contact-point velocity v_c = v_r + r_1 w_1 x n + r_2 w_2 x n, its tangential part
 * v_rt = v_c - (v_c.n) n, J_t = max(mu J_n, -(2/7)(1+e) m_r |v_rt|), t = v_rt/|v_rt|),
 * from each particle's own side (it is particle 1, its partner particle 2, n from 1
 * to 2). Readings: I = (2/5) m r^2 (solid sphere; the paper does not state I); the
 * two rotational terms of v_c are added in the order of the particles' ids (lower
 * first), so both sides see the same bits up to sign; |v_rt| = 0 gives no tangential
 * impulse; I (w' - w) = r (n x J) = r J_t (n x t). Positions as or_respond_advance. */
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

void or_respond_advance_rot(int64_t n, double* x, double* v, double* w, const double* r, const double* m,
                            const int32_t* id, const int64_t* partner, const double* tc, double e, double mu,
                            double dt) {
  double* xn = (double*)malloc(sizeof(double) * (size_t)(9 * n > 0 ? 9 * n : 1));
  if (!xn) return;
  double* vn = xn + 3 * n;
  double* wn = xn + 6 * n;
  for (int64_t i = 0; i < n; ++i) {
    int64_t j = partner[i];
    if (j < 0) {
      for (int k = 0; k < 3; ++k) {
        vn[k * n + i] = v[k * n + i];
        wn[k * n + i] = w[k * n + i];
        xn[k * n + i] = x[k * n + i] + dt * v[k * n + i];
      }
      continue;
    }
    const double t = tc[i];
    double dx[3], dv[3], s[3], nrm[3];
    for (int k = 0; k < 3; ++k) {
      dx[k] = minimg(x[k * n + i] - x[k * n + j]);
      dv[k] = v[k * n + i] - v[k * n + j];
    }
    for (int k = 0; k < 3; ++k) s[k] = dx[k] + t * dv[k];
    const double sl = sqrt((s[0] * s[0] + s[1] * s[1]) + s[2] * s[2]);
    for (int k = 0; k < 3; ++k) nrm[k] = -s[k] / sl;
    const double vrn = (dv[0] * nrm[0] + dv[1] * nrm[1]) + dv[2] * nrm[2];
    const double mr = (m[i] * m[j]) / (m[i] + m[j]);
    const double Jn = -mr * (1.0 + e) * vrn;
    /* contact-point velocity, rotational terms in id order */
    const int64_t lo = id[i] < id[j] ? i : j, hi = id[i] < id[j] ? j : i;
    double wl[3], wh[3], cl[3], ch[3], vc[3];
    for (int k = 0; k < 3; ++k) {
      wl[k] = w[k * n + lo];
      wh[k] = w[k * n + hi];
    }
    cross3(wl, nrm, cl);
    cross3(wh, nrm, ch);
    for (int k = 0; k < 3; ++k) vc[k] = (dv[k] + r[lo] * cl[k]) + r[hi] * ch[k];
    const double vcn = (vc[0] * nrm[0] + vc[1] * nrm[1]) + vc[2] * nrm[2];
    double vt[3];
    for (int k = 0; k < 3; ++k) vt[k] = vc[k] - vcn * nrm[k];
    const double vtl = sqrt((vt[0] * vt[0] + vt[1] * vt[1]) + vt[2] * vt[2]);
    double Jt = 0.0, tv[3] = {0.0, 0.0, 0.0};
    if (vtl > 0.0) {
      const double slide = mu * Jn, stick = -(2.0 / 7.0) * (1.0 + e) * mr * vtl;
      Jt = slide > stick ? slide : stick;
      for (int k = 0; k < 3; ++k) tv[k] = vt[k] / vtl;
    }
    const double gn = Jn / m[i], gt = Jt / m[i];
    double nt[3];
    cross3(nrm, tv, nt);
    const double inertia = 0.4 * m[i] * r[i] * r[i];
    const double gw = (r[i] * Jt) / inertia;
    for (int k = 0; k < 3; ++k) {
      const double vold = v[k * n + i];
      const double vnew = (vold + gn * nrm[k]) + gt * tv[k];
      vn[k * n + i] = vnew;
      wn[k * n + i] = w[k * n + i] + gw * nt[k];
      xn[k * n + i] = (x[k * n + i] + t * vold) + (dt - t) * vnew;
    }
  }
  for (int64_t a = 0; a < 3 * n; ++a) {
    v[a] = vn[a];
    w[a] = wn[a];
    x[a] = wrap01(xn[a]);
  }
  free(xn);
}

/* ---------------------------------------------------------- first-found pair selection */

/* Morton (Z-order) code of a cell: bit b of cx, cy, cz goes to bit 3b, 3b+1, 3b+2. */
static uint64_t morton3(uint64_t cx, uint64_t cy, uint64_t cz) {
  uint64_t code = 0;
  for (int b = 0; b < 21; ++b)
    code |= (((cx >> b) & 1u) << (3 * b)) | (((cy >> b) & 1u) << (3 * b + 1)) | (((cz >> b) & 1u) << (3 * b + 2));
  return code;
}

typedef struct {
  uint64_t key;
  int64_t idx;
} keyed_t;

static int cmp_keyed(const void* a, const void* b) {
  const keyed_t* x = (const keyed_t*)a;
  const keyed_t* y = (const keyed_t*)b;
  return x->key < y->key ? -1 : (x->key > y->key ? 1 : 0);
}

int64_t or_collide_step_sfc(int64_t n, double* x, double* v, const double* r, const double* m, const int32_t* id,
                            double e, double dt, int64_t ncell, int64_t* partner, double* tc) {
  int64_t cap = n > 16 ? 4 * n : 64;
  int64_t* ci = NULL;
  int64_t* cj = NULL;
  double* ct = NULL;
  int64_t nc = 0;
  for (;;) {
    ci = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    cj = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    ct = (double*)malloc(sizeof(double) * (size_t)cap);
    if (!ci || !cj || !ct) { free(ci); free(cj); free(ct); return -1; }
    nc = or_candidates_cells(n, x, v, r, dt, cap, ci, cj, ct);
    if (nc < 0) { free(ci); free(cj); free(ct); return -1; }
    if (nc <= cap) break;
    free(ci); free(cj); free(ct);
    cap = nc;
  }
  /* rank of every particle along the curve: (Morton code of its cell, id) */
  uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  keyed_t* order = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)(n > 0 ? n : 1));
  /* every particle's candidates, ordered by the partner's rank */
  keyed_t* adj = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)(2 * nc > 0 ? 2 * nc : 1));
  double* adjt = (double*)malloc(sizeof(double) * (size_t)(2 * nc > 0 ? 2 * nc : 1));
  int64_t* off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!key || !order || !adj || !adjt || !off) {
    free(ci); free(cj); free(ct); free(key); free(order); free(adj); free(adjt); free(off);
    return -1;
  }
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t code = morton3((uint64_t)cell_of(x[i], ncell), (uint64_t)cell_of(x[n + i], ncell),
                                  (uint64_t)cell_of(x[2 * n + i], ncell));
    key[i] = (code << 32) | (uint32_t)id[i];
    order[i].key = key[i];
    order[i].idx = i;
    partner[i] = -1;
    tc[i] = INFINITY;
  }
  qsort(order, (size_t)n, sizeof(keyed_t), cmp_keyed);
  for (int64_t k = 0; k < nc; ++k) {
    off[ci[k] + 1]++;
    off[cj[k] + 1]++;
  }
  for (int64_t i = 0; i < n; ++i) off[i + 1] += off[i];
  {
    int64_t* fill = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!fill) { free(ci); free(cj); free(ct); free(key); free(order); free(adj); free(adjt); free(off); return -1; }
    for (int64_t k = 0; k < nc; ++k) {
      const int64_t a = ci[k], b = cj[k];
      int64_t pa = off[a] + fill[a]++, pb = off[b] + fill[b]++;
      adj[pa].key = key[b];
      adj[pa].idx = b;
      adjt[pa] = ct[k];
      adj[pb].key = key[a];
      adj[pb].idx = a;
      adjt[pb] = ct[k];
    }
    free(fill);
  }
  /* sort each particle's candidates by partner rank, carrying the contact times */
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t a = off[i] + 1; a < off[i + 1]; ++a) {
      const keyed_t kk = adj[a];
      const double tt = adjt[a];
      int64_t b = a - 1;
      while (b >= off[i] && adj[b].key > kk.key) {
        adj[b + 1] = adj[b];
        adjt[b + 1] = adjt[b];
        --b;
      }
      adj[b + 1] = kk;
      adjt[b + 1] = tt;
    }
  }
  /* visit the particles along the curve; each free one takes its first free candidate */
  int64_t pairs = 0;
  for (int64_t q = 0; q < n; ++q) {
    const int64_t i = order[q].idx;
    if (partner[i] >= 0) continue;
    for (int64_t a = off[i]; a < off[i + 1]; ++a) {
      const int64_t j = adj[a].idx;
      if (partner[j] >= 0) continue;
      partner[i] = j;
      partner[j] = i;
      tc[i] = tc[j] = adjt[a];
      ++pairs;
      break;
    }
  }
  free(ci); free(cj); free(ct); free(key); free(order); free(adj); free(adjt); free(off);
  or_respond_advance(n, x, v, m, partner, tc, e, dt);
  return pairs;
}

int64_t or_collide_step(int64_t n, double* x, double* v, const double* r, const double* m, const int32_t* id,
                        double e, double dt, int method, int64_t* partner, double* tc) {
  int64_t cap = n > 16 ? 4 * n : 64;
  for (;;) {
    int64_t* ci = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    int64_t* cj = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    double* ct = (double*)malloc(sizeof(double) * (size_t)cap);
    if (!ci || !cj || !ct) { free(ci); free(cj); free(ct); return -1; }
    int64_t nc = method == 1 ? or_candidates_bruteforce(n, x, v, r, dt, cap, ci, cj, ct)
                             : or_candidates_cells(n, x, v, r, dt, cap, ci, cj, ct);
    if (nc < 0) { free(ci); free(cj); free(ct); return -1; }
    if (nc > cap) { free(ci); free(cj); free(ct); cap = nc; continue; }
    int64_t pairs = or_match_greedy(n, id, nc, ci, cj, ct, partner, tc);
    free(ci);
    free(cj);
    free(ct);
    if (pairs < 0) return -1;
    or_respond_advance(n, x, v, m, partner, tc, e, dt);
    return pairs;
  }
}

/* ------------------------------------------------------------------ projection */

void or_mesh_map(const double xi[3], double amp, double X[3], double* detJ) {
  const double tp = 6.283185307179586476925286766559;
  double s[3], c[3];
  for (int k = 0; k < 3; ++k) { s[k] = sin(tp * xi[k]); c[k] = cos(tp * xi[k]); }
  X[0] = xi[0] + amp * s[1] * s[2];
  X[1] = xi[1] + amp * s[2] * s[0];
  X[2] = xi[2] + amp * s[0] * s[1];
  /* D Phi = I + amp*2pi*[[0, c1 s2, s1 c2], [c0 s2, 0, s0 c2], [c0 s1, s0 c1, 0]] */
  double g = amp * tp;
  double A[3][3] = {{1.0, g * c[1] * s[2], g * s[1] * c[2]},
                    {g * c[0] * s[2], 1.0, g * s[0] * c[2]},
                    {g * c[0] * s[1], g * s[0] * c[1], 1.0}};
  *detJ = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
          A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

/* Neumaier's improvement of Kahan summation: s + c carries the running sum. */
static void neu_add(double* s, double* c, double t) {
  double u = *s + t;
  if (fabs(*s) >= fabs(t))
    *c += (*s - u) + t;
  else
    *c += (t - u) + *s;
  *s = u;
}

/* 1-D node indices (e*n1 + i) whose logical coordinate lies within `rad` of y
 * in the periodic minimum image; a plain scan over all ne*n1 1-D nodes. */
static int near_nodes(double y, double rad, int ne, int n1, const double* eta, int* out) {
  int cnt = 0;
  double h = 1.0 / ne;
  for (int e = 0; e < ne; ++e)
    for (int i = 0; i < n1; ++i) {
      double X = (e + 0.5 * (eta[i] + 1.0)) * h;
      if (fabs(minimg(X - y)) <= rad) out[cnt++] = e * n1 + i;
    }
  return cnt;
}

/* Visit every Gauss node within the cutoff of particle xp: pass 0 adds
 * W_g K(X_g - xp) to the Neumaier pair (zs, zc); pass 1 adds q_c K / zp to
 * node g of every component c. */
typedef struct {
  int ne, n1;
  int64_t nodes;
  double h, rc, inv2s2, amp;
  int cutoff_kind;
  const double *eta, *w;
  int *lx, *ly, *lz;
  double* field;
  double* comp;
} proj_ctx;

static void visit_support(const proj_ctx* P, const double xp[3], int pass, double* zs, double* zc, double zp,
                          const double qc[4]) {
  int n1 = P->n1, ne = P->ne;
  double rad = P->rc + fabs(P->amp);
  int nx = near_nodes(xp[0], rad, ne, n1, P->eta, P->lx);
  int ny = near_nodes(xp[1], rad, ne, n1, P->eta, P->ly);
  int nz = near_nodes(xp[2], rad, ne, n1, P->eta, P->lz);
  double hh = 0.5 * P->h;
  for (int c3 = 0; c3 < nz; ++c3)
    for (int b3 = 0; b3 < ny; ++b3)
      for (int a3 = 0; a3 < nx; ++a3) {
        int gx = P->lx[a3], gy = P->ly[b3], gz = P->lz[c3];
        int ex = gx / n1, i = gx % n1, ey = gy / n1, j = gy % n1, ez = gz / n1, k = gz % n1;
        double xi[3] = {(ex + 0.5 * (P->eta[i] + 1.0)) * P->h, (ey + 0.5 * (P->eta[j] + 1.0)) * P->h,
                        (ez + 0.5 * (P->eta[k] + 1.0)) * P->h};
        double X[3], detJ = 1.0;
        if (P->amp != 0.0) {
          or_mesh_map(xi, P->amp, X, &detJ);
        } else {
          X[0] = xi[0];
          X[1] = xi[1];
          X[2] = xi[2];
        }
        double d0 = minimg(X[0] - xp[0]), d1 = minimg(X[1] - xp[1]), d2 = minimg(X[2] - xp[2]);
        double d2s = (d0 * d0 + d1 * d1) + d2 * d2;
        if (P->cutoff_kind == 0) {
          if (!(fabs(d0) <= P->rc && fabs(d1) <= P->rc && fabs(d2) <= P->rc)) continue;
        } else {
          if (!(d2s <= P->rc * P->rc)) continue;
        }
        double K = exp(-d2s * P->inv2s2);
        if (pass == 0) {
          double W = P->w[i] * P->w[j] * P->w[k] * hh * hh * hh * detJ;
          neu_add(zs, zc, W * K);
        } else {
          double wk = K / zp;
          int64_t e = ((int64_t)ez * ne + ey) * ne + ex;
          int64_t base = e * 4 * P->nodes + ((int64_t)k * n1 + j) * n1 + i;
          for (int cc = 0; cc < 4; ++cc) {
            int64_t g = base + (int64_t)cc * P->nodes;
            neu_add(&P->field[g], &P->comp[g], qc[cc] * wk);
          }
        }
      }
}

/* Reading: the kernel K(d) = exp(-|d|^2/(2 sigma^2)) is cut at cutoff_sigmas*sigma
 * (box or sphere, inclusive); the discrete normalisation Z_p makes each particle's
 * quadrature-weighted deposit sum to its source, the Gaussian counterpart of the
 * denominator of the IDW deposition in Sec. 2.3. */
int or_project(int64_t n, const double* x, const double* q, int ne, int degree, double sigma, double cutoff_sigmas,
               int cutoff_kind, double amp, double* field, double* Z) {
  if (n < 0 || ne < 1 || degree < 0 || degree > 15 || !(sigma > 0.0) || !(cutoff_sigmas > 0.0)) return 1;
  if (cutoff_kind != 0 && cutoff_kind != 1) return 1;
  if (amp != 0.0 && cutoff_kind != 1) return 1;
  int n1 = degree + 1;
  double eta[16], w[16];
  if (or_gauss_legendre(n1, eta, w)) return 1;
  proj_ctx P;
  P.ne = ne;
  P.n1 = n1;
  P.nodes = (int64_t)n1 * n1 * n1;
  P.h = 1.0 / ne;
  P.rc = cutoff_sigmas * sigma;
  P.inv2s2 = 1.0 / (2.0 * sigma * sigma);
  P.amp = amp;
  P.cutoff_kind = cutoff_kind;
  P.eta = eta;
  P.w = w;
  int64_t nf = (int64_t)ne * ne * ne * 4 * P.nodes;
  P.lx = (int*)malloc(sizeof(int) * (size_t)(ne * n1));
  P.ly = (int*)malloc(sizeof(int) * (size_t)(ne * n1));
  P.lz = (int*)malloc(sizeof(int) * (size_t)(ne * n1));
  P.comp = (double*)calloc((size_t)nf, sizeof(double));
  P.field = field;
  if (!P.lx || !P.ly || !P.lz || !P.comp) {
    free(P.lx); free(P.ly); free(P.lz); free(P.comp);
    return 2;
  }
  for (int64_t a = 0; a < nf; ++a) field[a] = 0.0;
  for (int64_t p = 0; p < n; ++p) {
    double xp[3] = {x[p], x[n + p], x[2 * n + p]};
    double qc[4] = {q[p], q[n + p], q[2 * n + p], q[3 * n + p]};
    double zs = 0.0, zc = 0.0;
    visit_support(&P, xp, 0, &zs, &zc, 0.0, qc);
    double zp = zs + zc;
    if (Z) Z[p] = zp;
    if (zp > 0.0) visit_support(&P, xp, 1, NULL, NULL, zp, qc);
  }
  for (int64_t a = 0; a < nf; ++a) field[a] += P.comp[a];
  free(P.lx);
  free(P.ly);
  free(P.lz);
  free(P.comp);
  return 0;
}

/* ------------------------------------------------------------------ mixed storage */

int64_t or_collide_step_cellrel(int64_t n, int32_t nc, int32_t* cell, float* o, float* v, const float* r,
                                const float* m, const int32_t* id, double e, double dt, int64_t* partner,
                                double* tc) {
  const double L = (double)nc;
  /* exact FP64 cell-unit copies: x = c + o, v_c = v nc */
  double* x = (double*)malloc(sizeof(double) * (size_t)(3 * n > 0 ? 3 * n : 1));
  double* vc = (double*)malloc(sizeof(double) * (size_t)(3 * n > 0 ? 3 * n : 1));
  double* vn = (double*)malloc(sizeof(double) * (size_t)(3 * n > 0 ? 3 * n : 1));
  int64_t cap = n > 16 ? 4 * n : 64;
  int64_t *ci = NULL, *cj = NULL;
  double* ct = NULL;
  if (!x || !vc || !vn) { free(x); free(vc); free(vn); return -1; }
  for (int64_t i = 0; i < n; ++i) {
    int32_t cl = cell[i];
    int32_t c3[3] = {cl % nc, (cl / nc) % nc, cl / (nc * nc)};
    for (int k = 0; k < 3; ++k) {
      x[k * n + i] = (double)c3[k] + (double)o[k * n + i];
      vc[k * n + i] = (double)v[k * n + i] * L;
    }
  }
  /* candidates by brute force over all pairs (plain; the mixed tests use small n) */
  int64_t cnt;
  for (;;) {
    ci = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    cj = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    ct = (double*)malloc(sizeof(double) * (size_t)cap);
    if (!ci || !cj || !ct) { free(ci); free(cj); free(ct); free(x); free(vc); free(vn); return -1; }
    cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
      double xi[3] = {x[i], x[n + i], x[2 * n + i]};
      double vi[3] = {vc[i], vc[n + i], vc[2 * n + i]};
      for (int64_t j = i + 1; j < n; ++j) {
        double xj[3] = {x[j], x[n + j], x[2 * n + j]};
        double vj[3] = {vc[j], vc[n + j], vc[2 * n + j]};
        double R = ((double)r[i] + (double)r[j]) * L;
        double t = contact_time_box(xi, xj, vi, vj, R, dt, L);
        if (t <= dt) {
          if (cnt < cap) { ci[cnt] = i; cj[cnt] = j; ct[cnt] = t; }
          ++cnt;
        }
      }
    }
    if (cnt <= cap) break;
    free(ci); free(cj); free(ct);
    cap = cnt;
  }
  int64_t pairs = or_match_greedy(n, id, cnt, ci, cj, ct, partner, tc);
  free(ci); free(cj); free(ct);
  if (pairs < 0) { free(x); free(vc); free(vn); return -1; }
  const float dtn = (float)(dt * L);
  for (int64_t i = 0; i < n; ++i) {
    int32_t cl = cell[i];
    int32_t c3[3] = {cl % nc, (cl / nc) % nc, cl / (nc * nc)};
    int64_t j = partner[i];
    if (j < 0) {
      /* free flight in FP32 cell units with a carry */
      for (int k = 0; k < 3; ++k) {
        float on = o[k * n + i] + dtn * v[k * n + i];
        if (on >= 1.0f) {
          on = on - 1.0f;
          c3[k] = c3[k] + 1 == nc ? 0 : c3[k] + 1;
        } else if (on < 0.0f) {
          float up = on + 1.0f;
          if (up == 1.0f) {
            on = 0.0f;
          } else {
            on = up;
            c3[k] = c3[k] == 0 ? nc - 1 : c3[k] - 1;
          }
        }
        o[k * n + i] = on;
      }
    } else {
      /* FP64 response: physical velocities, cell-unit positions */
      double t = tc[i];
      double dx[3], dvc[3], dv[3], s3[3], nr[3];
      for (int k = 0; k < 3; ++k) {
        dx[k] = minimg_box(x[k * n + i] - x[k * n + j], L);
        dvc[k] = vc[k * n + i] - vc[k * n + j];
        dv[k] = (double)v[k * n + i] - (double)v[k * n + j];
      }
      for (int k = 0; k < 3; ++k) s3[k] = dx[k] + t * dvc[k];
      double sl = sqrt((s3[0] * s3[0] + s3[1] * s3[1]) + s3[2] * s3[2]);
      for (int k = 0; k < 3; ++k) nr[k] = -s3[k] / sl;
      double vrn = (dv[0] * nr[0] + dv[1] * nr[1]) + dv[2] * nr[2];
      double mi = (double)m[i], mj = (double)m[j];
      double mr = (mi * mj) / (mi + mj);
      double J = -mr * (1.0 + e) * vrn;
      double gi = J / mi;
      for (int k = 0; k < 3; ++k) {
        double vold = (double)v[k * n + i];
        double vnew = vold + gi * nr[k];
        double y = (x[k * n + i] + t * vc[k * n + i]) + (dt - t) * (vnew * L);
        if (y < 0.0) y += L;
        else if (y >= L) y -= L;
        int32_t cq = (int32_t)floor(y);
        if (cq < 0) cq = 0;
        if (cq > nc - 1) cq = nc - 1;
        float oq = (float)(y - (double)cq);
        if (oq >= 1.0f) {
          oq = 0.0f;
          cq = cq + 1 == nc ? 0 : cq + 1;
        }
        c3[k] = cq;
        o[k * n + i] = oq;
        vn[k * n + i] = vnew;
      }
    }
    cell[i] = (c3[2] * nc + c3[1]) * nc + c3[0];
  }
  /* velocities are stored only after every pair has read the old ones */
  for (int64_t i = 0; i < n; ++i)
    if (partner[i] >= 0)
      for (int k = 0; k < 3; ++k) v[k * n + i] = (float)vn[k * n + i];
  free(x);
  free(vc);
  free(vn);
  return pairs;
}

/* ------------------------------------------------------------------ adjoint */

int or_collide_replay(int64_t n, double* x, double* v, const double* r, const double* m, const int64_t* partner,
                      double e, double dt) {
  double* tc = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!tc) return -2;
  int bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    tc[i] = INFINITY;
    int64_t j = partner[i];
    if (j < 0) continue;
    double xi[3], xj[3], vi[3], vj[3];
    load3(x, n, i, xi);
    load3(x, n, j, xj);
    load3(v, n, i, vi);
    load3(v, n, j, vj);
    double t = or_contact_time(xi, xj, vi, vj, r[i], r[j], dt);
    if (!(t <= dt)) bad = 1;
    tc[i] = t;
  }
  if (!bad) or_respond_advance(n, x, v, m, partner, tc, e, dt);
  free(tc);
  return bad ? -1 : 0;
}

static double dot3(const double a[3], const double b[3]) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

int or_collide_adjoint(int64_t n, const double* x, const double* v, const double* r, const double* m,
                       const int64_t* partner, double e, double dt, const double* gx_out, const double* gv_out,
                       double* gx_in, double* gv_in) {
  /* free flight: x' = x + dt v, v' = v */
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      gx_in[k * n + i] = gx_out[k * n + i];
      gv_in[k * n + i] = gv_out[k * n + i] + dt * gx_out[k * n + i];
    }
  for (int64_t i = 0; i < n; ++i) {
    int64_t j = partner[i];
    if (j < 0 || j < i) continue; /* each pair once, from its lower index */
    double xi[3], xj[3], vi[3], vj[3];
    load3(x, n, i, xi);
    load3(x, n, j, xj);
    load3(v, n, i, vi);
    load3(v, n, j, vj);
    double t = or_contact_time(xi, xj, vi, vj, r[i], r[j], dt);
    if (!(t <= dt)) return -1;
    /* forward intermediates */
    double dx[3], dv[3], s[3], nrm[3], vin[3], vjn[3];
    for (int k = 0; k < 3; ++k) {
      dx[k] = minimg(xi[k] - xj[k]);
      dv[k] = vi[k] - vj[k];
      s[k] = dx[k] + t * dv[k];
    }
    double sl = sqrt(dot3(s, s));
    for (int k = 0; k < 3; ++k) nrm[k] = -s[k] / sl;
    double vrn = dot3(dv, nrm);
    double mr = (m[i] * m[j]) / (m[i] + m[j]);
    double J = -mr * (1.0 + e) * vrn;
    for (int k = 0; k < 3; ++k) {
      vin[k] = vi[k] + (J / m[i]) * nrm[k];
      vjn[k] = vj[k] - (J / m[j]) * nrm[k];
    }
    double Xi[3], Xj[3], Vi[3], Vj[3];
    for (int k = 0; k < 3; ++k) {
      Xi[k] = gx_out[k * n + i];
      Xj[k] = gx_out[k * n + j];
      Vi[k] = gv_out[k * n + i];
      Vj[k] = gv_out[k * n + j];
    }
    /* reverse sweep; the free-flight initialisation above is replaced for i and j */
    double gxi[3], gxj[3], gvi[3], gvj[3], gdx[3] = {0, 0, 0}, gdv[3] = {0, 0, 0}, gn[3] = {0, 0, 0};
    double gt = 0.0, gJ = 0.0;
    double Vit[3], Vjt[3];
    for (int k = 0; k < 3; ++k) {
      /* x_i' = x_i + t v_i + (dt - t) v_i' */
      gxi[k] = Xi[k];
      gvi[k] = t * Xi[k];
      Vit[k] = Vi[k] + (dt - t) * Xi[k];
      gt += Xi[k] * (vi[k] - vin[k]);
      gxj[k] = Xj[k];
      gvj[k] = t * Xj[k];
      Vjt[k] = Vj[k] + (dt - t) * Xj[k];
      gt += Xj[k] * (vj[k] - vjn[k]);
    }
    /* v_i' = v_i + (J/m_i) n, v_j' = v_j - (J/m_j) n */
    for (int k = 0; k < 3; ++k) {
      gvi[k] += Vit[k];
      gvj[k] += Vjt[k];
      gn[k] += (J / m[i]) * Vit[k] - (J / m[j]) * Vjt[k];
    }
    gJ = dot3(Vit, nrm) / m[i] - dot3(Vjt, nrm) / m[j];
    /* J = -m_r (1 + e) v_rn, v_rn = dv . n */
    double gvrn = -mr * (1.0 + e) * gJ;
    for (int k = 0; k < 3; ++k) {
      gdv[k] += gvrn * nrm[k];
      gn[k] += gvrn * dv[k];
    }
    /* n = -s/|s|: gs = -(gn - nh (nh . gn))/|s| with nh = s/|s| */
    double nh[3] = {s[0] / sl, s[1] / sl, s[2] / sl};
    double pg = dot3(nh, gn);
    double gs[3];
    for (int k = 0; k < 3; ++k) gs[k] = -(gn[k] - nh[k] * pg) / sl;
    /* s = dx + t dv */
    for (int k = 0; k < 3; ++k) {
      gdx[k] += gs[k];
      gdv[k] += t * gs[k];
    }
    gt += dot3(gs, dv);
    /* t from |dx + t dv| = R: dt/d(dx) = -s/(s.dv), dt/d(dv) = -t s/(s.dv) */
    double sdv = dot3(s, dv);
    for (int k = 0; k < 3; ++k) {
      gdx[k] += gt * (-s[k] / sdv);
      gdv[k] += gt * (-t * s[k] / sdv);
    }
    for (int k = 0; k < 3; ++k) {
      gx_in[k * n + i] = gxi[k] + gdx[k];
      gx_in[k * n + j] = gxj[k] - gdx[k];
      gv_in[k * n + i] = gvi[k] + gdv[k];
      gv_in[k * n + j] = gvj[k] - gdv[k];
    }
  }
  return 0;
}

int or_project_adjoint(int64_t n, const double* x, const double* q, int ne, int degree, double sigma,
                       double cutoff_sigmas, int cutoff_kind, const double* G, double* gq, double* gx) {
  if (n < 0 || ne < 1 || degree < 0 || degree > 15 || !(sigma > 0.0)) return 1;
  int n1 = degree + 1;
  double eta[16], w[16];
  if (or_gauss_legendre(n1, eta, w)) return 1;
  int64_t nodes = (int64_t)n1 * n1 * n1;
  double h = 1.0 / ne, hh = 0.5 * h, rc = cutoff_sigmas * sigma, s2 = sigma * sigma;
  int* lx = (int*)malloc(sizeof(int) * (size_t)(ne * n1));
  int* ly = (int*)malloc(sizeof(int) * (size_t)(ne * n1));
  int* lz = (int*)malloc(sizeof(int) * (size_t)(ne * n1));
  if (!lx || !ly || !lz) { free(lx); free(ly); free(lz); return 2; }
  for (int64_t p = 0; p < n; ++p) {
    double xp[3] = {x[p], x[n + p], x[2 * n + p]};
    int nx = near_nodes(xp[0], rc, ne, n1, eta, lx);
    int ny = near_nodes(xp[1], rc, ne, n1, eta, ly);
    int nz = near_nodes(xp[2], rc, ne, n1, eta, lz);
    /* Z = sum W K, Z1 = sum W K d, S0 = sum a K, S1 = sum a K d, with a = sum_c G_c q_c */
    double Z = 0, Z1[3] = {0, 0, 0}, S0 = 0, S1[3] = {0, 0, 0}, GK[4] = {0, 0, 0, 0};
    for (int pass = 0; pass < 2; ++pass)
      for (int c3 = 0; c3 < nz; ++c3)
        for (int b3 = 0; b3 < ny; ++b3)
          for (int a3 = 0; a3 < nx; ++a3) {
            int gx_ = lx[a3], gy = ly[b3], gz = lz[c3];
            int ex = gx_ / n1, i = gx_ % n1, ey = gy / n1, j = gy % n1, ez = gz / n1, k = gz % n1;
            double X[3] = {(ex + 0.5 * (eta[i] + 1.0)) * h, (ey + 0.5 * (eta[j] + 1.0)) * h,
                           (ez + 0.5 * (eta[k] + 1.0)) * h};
            double d[3] = {minimg(X[0] - xp[0]), minimg(X[1] - xp[1]), minimg(X[2] - xp[2])};
            double d2s = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (cutoff_kind == 0) {
              if (!(fabs(d[0]) <= rc && fabs(d[1]) <= rc && fabs(d[2]) <= rc)) continue;
            } else if (!(d2s <= rc * rc)) {
              continue;
            }
            double K = exp(-d2s / (2.0 * s2));
            if (pass == 0) {
              double W = w[i] * w[j] * w[k] * hh * hh * hh;
              Z += W * K;
              for (int a = 0; a < 3; ++a) Z1[a] += W * K * d[a];
            } else {
              int64_t e = ((int64_t)ez * ne + ey) * ne + ex;
              int64_t base = e * 4 * nodes + ((int64_t)k * n1 + j) * n1 + i;
              double a = 0;
              for (int c = 0; c < 4; ++c) {
                double g = G[base + (int64_t)c * nodes];
                a += g * q[(int64_t)c * n + p];
                GK[c] += g * K;
              }
              S0 += a * K;
              for (int aa = 0; aa < 3; ++aa) S1[aa] += a * K * d[aa];
            }
          }
    for (int c = 0; c < 4; ++c) gq[(int64_t)c * n + p] = Z > 0 ? GK[c] / Z : 0.0;
    for (int a = 0; a < 3; ++a) gx[(int64_t)a * n + p] = Z > 0 ? (S1[a] / Z - S0 * Z1[a] / (Z * Z)) / s2 : 0.0;
  }
  free(lx);
  free(ly);
  free(lz);
  return 0;
}

/* ------------------------------------------------------------------ corner-node and Dirac deposition */

/* Trilinear weight of corner (dx, dy, dz) in {0,1}^3 of an element at reference
 * position xi in [-1,1]^3: prod_d (1 + s_d xi_d) / 2 with s_d = -1 for d = 0 and
 * +1 for d = 1, i.e. 1 at its own corner, 0 at the others. */
static double corner_weight(int dx, int dy, int dz, const double xi[3]) {
  const double a = dx ? 0.5 * (1.0 + xi[0]) : 0.5 * (1.0 - xi[0]);
  const double b = dy ? 0.5 * (1.0 + xi[1]) : 0.5 * (1.0 - xi[1]);
  const double c = dz ? 0.5 * (1.0 + xi[2]) : 0.5 * (1.0 - xi[2]);
  return a * b * c;
}

/* Element of a coordinate in [0,1) and the reference coordinate 2 (x ne - e) - 1. */
static int elem_ref(double y, int ne, double* xi) {
  int e = (int)floor(y * ne);
  if (e < 0) e = 0;
  if (e > ne - 1) e = ne - 1;
  *xi = 2.0 * (y * ne - e) - 1.0;
  return e;
}

static int64_t corner_node(int ex, int ey, int ez, int dx, int dy, int dz, int ne) {
  return ((int64_t)((ez + dz) % ne) * ne + (ey + dy) % ne) * ne + (ex + dx) % ne;
}

int or_project_idw(int64_t n, const double* x, const double* q, int ne, int degree, double* field) {
  if (n < 0 || ne < 1 || degree < 0 || degree > 15 || !field || (n > 0 && (!x || !q))) return 1;
  const int n1 = degree + 1, nodes = n1 * n1 * n1;
  const int64_t nel = (int64_t)ne * ne * ne;
  double eta[16], w[16];
  if (or_gauss_legendre(n1, eta, w)) return 1;
  const double h = 1.0 / ne, jac = 0.125 * h * h * h;
  double* S = (double*)calloc((size_t)(8 * nel + 2 * nel), sizeof(double)); /* [4][nel] sums + [4][nel] comp + V, Vc */
  if (!S) return 4;
  double* Sc = S + 4 * nel;
  double* V = S + 8 * nel;
  double* Vc = V + nel;
  /* node volumes: the quadrature of each corner's trilinear hat over the elements around it */
  for (int ez = 0; ez < ne; ++ez)
    for (int ey = 0; ey < ne; ++ey)
      for (int ex = 0; ex < ne; ++ex)
        for (int d = 0; d < 8; ++d)
          for (int k = 0; k < n1; ++k)
            for (int j = 0; j < n1; ++j)
              for (int i = 0; i < n1; ++i) {
                const double xg[3] = {eta[i], eta[j], eta[k]};
                const int64_t N = corner_node(ex, ey, ez, d & 1, (d >> 1) & 1, d >> 2, ne);
                neu_add(&V[N], &Vc[N], w[i] * w[j] * w[k] * jac * corner_weight(d & 1, (d >> 1) & 1, d >> 2, xg));
              }
  /* node sums of the sources */
  for (int64_t p = 0; p < n; ++p) {
    double xi[3];
    const int ex = elem_ref(x[p], ne, &xi[0]), ey = elem_ref(x[n + p], ne, &xi[1]), ez = elem_ref(x[2 * n + p], ne, &xi[2]);
    for (int d = 0; d < 8; ++d) {
      const int64_t N = corner_node(ex, ey, ez, d & 1, (d >> 1) & 1, d >> 2, ne);
      const double wt = corner_weight(d & 1, (d >> 1) & 1, d >> 2, xi);
      for (int c = 0; c < 4; ++c) neu_add(&S[c * nel + N], &Sc[c * nel + N], q[c * n + p] * wt);
    }
  }
  /* field at the Gauss nodes: trilinear interpolation of the corner densities */
  for (int ez = 0; ez < ne; ++ez)
    for (int ey = 0; ey < ne; ++ey)
      for (int ex = 0; ex < ne; ++ex) {
        const int64_t e = ((int64_t)ez * ne + ey) * ne + ex;
        for (int k = 0; k < n1; ++k)
          for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n1; ++i) {
              const double xg[3] = {eta[i], eta[j], eta[k]};
              for (int c = 0; c < 4; ++c) {
                double s = 0.0, sc = 0.0;
                for (int d = 0; d < 8; ++d) {
                  const int64_t N = corner_node(ex, ey, ez, d & 1, (d >> 1) & 1, d >> 2, ne);
                  const double dens = (S[c * nel + N] + Sc[c * nel + N]) / (V[N] + Vc[N]);
                  neu_add(&s, &sc, corner_weight(d & 1, (d >> 1) & 1, d >> 2, xg) * dens);
                }
                field[(e * 4 + c) * nodes + ((int64_t)k * n1 + j) * n1 + i] = s + sc;
              }
            }
      }
  free(S);
  return 0;
}

int or_project_dirac(int64_t n, const double* x, const double* q, int ne, int degree, double* field) {
  if (n < 0 || ne < 1 || degree < 0 || degree > 15 || !field || (n > 0 && (!x || !q))) return 1;
  const int n1 = degree + 1, nodes = n1 * n1 * n1;
  const int64_t nel = (int64_t)ne * ne * ne;
  double eta[16], w[16];
  if (or_gauss_legendre(n1, eta, w)) return 1;
  const double h = 1.0 / ne, jac = 0.125 * h * h * h;
  double* cmp = (double*)calloc((size_t)(nel * 4 * nodes), sizeof(double));
  if (!cmp) return 4;
  memset(field, 0, sizeof(double) * (size_t)(nel * 4 * nodes));
  for (int64_t p = 0; p < n; ++p) {
    int e3[3], i3[3];
    for (int a = 0; a < 3; ++a) {
      double xi;
      e3[a] = elem_ref(x[a * n + p], ne, &xi);
      /* nearest Gauss node along the axis; the lower index on a tie */
      int best = 0;
      for (int i = 1; i < n1; ++i)
        if (fabs(eta[i] - xi) < fabs(eta[best] - xi)) best = i;
      i3[a] = best;
    }
    const int64_t e = ((int64_t)e3[2] * ne + e3[1]) * ne + e3[0];
    const int g = (i3[2] * n1 + i3[1]) * n1 + i3[0];
    for (int c = 0; c < 4; ++c) {
      const int64_t o = (e * 4 + c) * nodes + g;
      neu_add(&field[o], &cmp[o], q[c * n + p]);
    }
  }
  for (int64_t e = 0; e < nel; ++e)
    for (int c = 0; c < 4; ++c)
      for (int k = 0; k < n1; ++k)
        for (int j = 0; j < n1; ++j)
          for (int i = 0; i < n1; ++i) {
            const int64_t o = (e * 4 + c) * nodes + ((int64_t)k * n1 + j) * n1 + i;
            field[o] = (field[o] + cmp[o]) / (w[i] * w[j] * w[k] * jac);
          }
  free(cmp);
  return 0;
}

/* ------------------------------------------------------------------ field at particles, drag sources */

/* Lagrange basis polynomial i of the nodes eta[0..n1) at xi: prod_{m != i} (xi - eta_m) / (eta_i - eta_m). */
static double lagrange(int n1, const double* eta, int i, double xi) {
  double num = 1.0, den = 1.0;
  for (int m = 0; m < n1; ++m) {
    if (m == i) continue;
    num *= xi - eta[m];
    den *= eta[i] - eta[m];
  }
  return num / den;
}

int or_eval_field(int64_t n, const double* x, const double* field, int ne, int degree, int nvar, double* out) {
  if (n < 0 || ne < 1 || degree < 0 || degree > 15 || nvar < 1 || (n > 0 && (!x || !field || !out))) return 1;
  const int n1 = degree + 1, nodes = n1 * n1 * n1;
  double eta[16], w[16];
  if (or_gauss_legendre(n1, eta, w)) return 1;
  for (int64_t p = 0; p < n; ++p) {
    double xi[3];
    const int ex = elem_ref(x[p], ne, &xi[0]), ey = elem_ref(x[n + p], ne, &xi[1]), ez = elem_ref(x[2 * n + p], ne, &xi[2]);
    const int64_t e = ((int64_t)ez * ne + ey) * ne + ex;
    double lx[16], ly[16], lz[16];
    for (int i = 0; i < n1; ++i) {
      lx[i] = lagrange(n1, eta, i, xi[0]);
      ly[i] = lagrange(n1, eta, i, xi[1]);
      lz[i] = lagrange(n1, eta, i, xi[2]);
    }
    for (int c = 0; c < nvar; ++c) {
      const double* U = field + (e * nvar + c) * nodes;
      double s = 0.0, sc = 0.0;
      for (int k = 0; k < n1; ++k)
        for (int j = 0; j < n1; ++j)
          for (int i = 0; i < n1; ++i) neu_add(&s, &sc, U[(k * n1 + j) * n1 + i] * (lx[i] * ly[j] * lz[k]));
      out[c * n + p] = s + sc;
    }
  }
  return 0;
}

void or_drag_sources(int64_t n, const double* v, const double* r, const double* fluid, double mu_f, double* q) {
  const double pi = 3.14159265358979323846;
  for (int64_t p = 0; p < n; ++p) {
    const double d = 2.0 * r[p];
    const double rho = fluid[p];
    double rel[3], F[3];
    for (int k = 0; k < 3; ++k) rel[k] = fluid[(k + 1) * n + p] - v[k * n + p];
    const double speed = sqrt((rel[0] * rel[0] + rel[1] * rel[1]) + rel[2] * rel[2]);
    const double re = rho * speed * d / mu_f;
    const double fd = 1.0 + 0.15 * pow(re, 0.687);
    const double coef = 3.0 * pi * mu_f * d * fd;
    for (int k = 0; k < 3; ++k) F[k] = coef * rel[k];
    for (int k = 0; k < 3; ++k) q[k * n + p] = -F[k];
    q[3 * n + p] = -((F[0] * v[p] + F[1] * v[n + p]) + F[2] * v[2 * n + p]);
  }
}
