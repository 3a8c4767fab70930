/*
 * Seeded synthetic particle workloads: sphere packings in the periodic unit cube.
 *
 * This file only draws inputs. It holds none of the collision or projection
 * arithmetic; both the CPU oracle and the CUDA path consume the arrays it writes.
 *
 * Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), one independent stream per
 * quantity: stream s of seed S starts at state S * 0x9E37... ^ hash(s).
 * Uniform doubles take the top 53 bits. Normals use the Box-Muller transform.
 *
 * Positions: random sequential addition (RSA). A uniform candidate centre is
 * rejected while it overlaps (or touches) a sphere already placed, measured with
 * the periodic minimum image; spheres are placed in the order their diameters
 * were drawn. A uniform hash grid with cell side >= the largest diameter keeps
 * each test to the 27 neighbouring cells.
 *
 * Large packings are placed by speculative batches with the same result as the
 * one-by-one process (see pcgen_rsa).
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared -pthread gen.c -lm
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

static uint64_t sm64_next(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint64_t stream_state(uint64_t seed, uint64_t stream) {
  uint64_t s = seed ^ (stream * 0xD1B54A32D192ED03ull);
  /* decorrelate neighbouring seeds/streams */
  (void)sm64_next(&s);
  (void)sm64_next(&s);
  return s;
}

/* uniform in [0,1) with 53 random bits */
static double u01(uint64_t* s) { return (double)(sm64_next(s) >> 11) * 0x1.0p-53; }

/* uniform in (0,1] */
static double u01_open0(uint64_t* s) { return ((double)(sm64_next(s) >> 11) + 1.0) * 0x1.0p-53; }

static const double kTwoPi = 6.283185307179586476925286766559;

/* Fill out[0..n) with i.i.d. N(0, scale^2) from stream `stream`. */
int pcgen_normal(int64_t n, uint64_t seed, uint64_t stream, double scale, double* out) {
  if (n < 0 || !out) return 1;
  uint64_t s = stream_state(seed, stream);
  for (int64_t i = 0; i < n; i += 2) {
    double u1 = u01_open0(&s), u2 = u01(&s);
    double rad = sqrt(-2.0 * log(u1));
    out[i] = scale * rad * cos(kTwoPi * u2);
    if (i + 1 < n) out[i + 1] = scale * rad * sin(kTwoPi * u2);
  }
  return 0;
}

/* Fill out[0..n) with i.i.d. U[lo, hi). */
int pcgen_uniform(int64_t n, uint64_t seed, uint64_t stream, double lo, double hi, double* out) {
  if (n < 0 || !out) return 1;
  uint64_t s = stream_state(seed, stream);
  for (int64_t i = 0; i < n; ++i) out[i] = lo + (hi - lo) * u01(&s);
  return 0;
}

/* Velocities of fixed magnitude `speed` with isotropic random directions, SoA v[3][n]. */
int pcgen_fixed_speed(int64_t n, uint64_t seed, uint64_t stream, double speed, double* v) {
  if (n < 0 || !v) return 1;
  uint64_t s = stream_state(seed, stream);
  for (int64_t i = 0; i < n; ++i) {
    double cz = 2.0 * u01(&s) - 1.0, ph = kTwoPi * u01(&s);
    double sz = sqrt(fmax(0.0, 1.0 - cz * cz));
    v[i] = speed * sz * cos(ph);
    v[n + i] = speed * sz * sin(ph);
    v[2 * n + i] = speed * cz;
  }
  return 0;
}

/*
 * Diameters: kind 0 constant p0; kind 1 uniform [p0, p1]; kind 2 lognormal with
 * median p0 and log-standard-deviation p1, clipped to [p2, p3] when p2 > 0.
 */
int pcgen_diameters(int64_t n, uint64_t seed, int kind, double p0, double p1, double p2, double p3, double* d) {
  if (n < 0 || !d) return 1;
  uint64_t s = stream_state(seed, 2);
  for (int64_t i = 0; i < n; ++i) {
    double di;
    if (kind == 0) {
      di = p0;
    } else if (kind == 1) {
      di = p0 + (p1 - p0) * u01(&s);
    } else if (kind == 2) {
      double u1 = u01_open0(&s), u2 = u01(&s);
      double z = sqrt(-2.0 * log(u1)) * cos(kTwoPi * u2);
      di = p0 * exp(p1 * z);
      if (p2 > 0.0) di = fmin(fmax(di, p2), p3);
    } else {
      return 2;
    }
    d[i] = di;
  }
  return 0;
}

static double minimg(double a) {
  if (a > 0.5) return a - 1.0;
  if (a < -0.5) return a + 1.0;
  return a;
}

/*
 * RSA placement of n spheres of radii r[] (already drawn) in the periodic unit
 * cube. Writes centres x[3][n] (SoA). Returns 0 on success, 3 when the number of
 * rejected candidates exceeds max_reject (the packing jammed), 1 on bad input,
 * 4 when memory runs out.
 */
/* A placed sphere as the neighbour search reads it: centre, radius and the next
 * sphere of its grid cell in one record, so that each comparison touches one
 * cache line. */
typedef struct {
  double x, y, z, r;
  int64_t next;
} rsa_node;

/* Candidate centres are drawn from the stream in a fixed order whatever the
 * outcomes, so they are drawn kAhead ahead of their test: the grid rows a
 * candidate will read are prefetched when it is drawn, the first sphere of each
 * of its cells kNodeAhead candidates before its test. Prefetching changes no
 * result. */
enum { kAhead = 16, kNodeAhead = 6 };

static int64_t cell_index(double p, int64_t ng) {
  int64_t c = (int64_t)(p * ng);
  return c >= ng ? ng - 1 : c;
}

/* a + d for a in [0, ng), d in {-1, 0, 1}, wrapped periodically */
static int64_t wrap_step(int64_t a, int64_t d, int64_t ng) {
  a += d;
  return a < 0 ? a + ng : (a >= ng ? a - ng : a);
}

static int rsa_sequential(int64_t n, uint64_t seed, const double* r, double* x, int64_t max_reject,
                          int64_t* rejects_out) {
  if (n < 0 || !r || !x) return 1;
  if (n == 0) return 0;
  double rmax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(r[i] > 0.0) || r[i] >= 0.25) return 1;
    if (r[i] > rmax) rmax = r[i];
  }
  /* grid side >= 2*rmax, at most 2^30 cells */
  int64_t ng = (int64_t)floor(1.0 / (2.0 * rmax * (1.0 + 1e-9)));
  if (ng < 1) ng = 1;
  while (ng > 1 && ng * ng * ng > ((int64_t)1 << 30)) --ng;
  int64_t ncell = ng * ng * ng;
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
  rsa_node* node = (rsa_node*)malloc(sizeof(rsa_node) * (size_t)n);
  if (!head || !node) { free(head); free(node); return 4; }
  for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
  uint64_t s = stream_state(seed, 1);
  int64_t rejects = 0;
  int span = ng >= 3 ? 1 : 0; /* ng < 3: every cell is a neighbour; scan all once */
  double ring[kAhead][3];
  int64_t drawn = 0, used = 0;
  for (int64_t i = 0; i < n; ++i) {
    const double ri = r[i];
    for (;;) {
      while (drawn < used + kAhead) {
        double* c = ring[drawn % kAhead];
        c[0] = u01(&s);
        c[1] = u01(&s);
        c[2] = u01(&s);
        if (span) {
          const int64_t cx = cell_index(c[0], ng), cy = cell_index(c[1], ng), cz = cell_index(c[2], ng);
          for (int64_t dz = -1; dz <= 1; ++dz)
            for (int64_t dy = -1; dy <= 1; ++dy) {
              const int64_t row = (wrap_step(cz, dz, ng) * ng + wrap_step(cy, dy, ng)) * ng;
              __builtin_prefetch(&head[row + wrap_step(cx, -1, ng)]);
              __builtin_prefetch(&head[row + wrap_step(cx, 1, ng)]);
            }
        }
        ++drawn;
      }
      if (span && drawn > used + kNodeAhead) {
        const double* c = ring[(used + kNodeAhead) % kAhead];
        const int64_t cx = cell_index(c[0], ng), cy = cell_index(c[1], ng), cz = cell_index(c[2], ng);
        for (int64_t dz = -1; dz <= 1; ++dz)
          for (int64_t dy = -1; dy <= 1; ++dy)
            for (int64_t dx = -1; dx <= 1; ++dx) {
              const int64_t j = head[(wrap_step(cz, dz, ng) * ng + wrap_step(cy, dy, ng)) * ng + wrap_step(cx, dx, ng)];
              if (j >= 0) __builtin_prefetch(&node[j]);
            }
      }
      const double* cand = ring[used % kAhead];
      const double px = cand[0], py = cand[1], pz = cand[2];
      ++used;
      const int64_t cx = cell_index(px, ng), cy = cell_index(py, ng), cz = cell_index(pz, ng);
      int ok = 1;
      int64_t lo = span ? -1 : 0, hi = span ? 1 : ng - 1;
      for (int64_t dz = lo; dz <= hi && ok; ++dz)
        for (int64_t dy = lo; dy <= hi && ok; ++dy)
          for (int64_t dx = lo; dx <= hi && ok; ++dx) {
            int64_t ax = span ? wrap_step(cx, dx, ng) : dx;
            int64_t ay = span ? wrap_step(cy, dy, ng) : dy;
            int64_t az = span ? wrap_step(cz, dz, ng) : dz;
            for (int64_t j = head[(az * ng + ay) * ng + ax]; j >= 0; j = node[j].next) {
              const rsa_node* q = &node[j];
              double ddx = minimg(px - q->x), ddy = minimg(py - q->y), ddz = minimg(pz - q->z);
              double rr = ri + q->r;
              if (ddx * ddx + ddy * ddy + ddz * ddz <= rr * rr) { ok = 0; break; }
            }
          }
      if (ok) {
        x[i] = px; x[n + i] = py; x[2 * n + i] = pz;
        int64_t c = (cz * ng + cy) * ng + cx;
        node[i].x = px;
        node[i].y = py;
        node[i].z = pz;
        node[i].r = ri;
        node[i].next = head[c];
        head[c] = i;
        break;
      }
      if (++rejects > max_reject) { free(head); free(node); if (rejects_out) *rejects_out = rejects; return 3; }
    }
  }
  free(head);
  free(node);
  if (rejects_out) *rejects_out = rejects;
  return 0;
}

/* ---------------------------------------------------------- batched placement
 *
 * The candidate centres come from the stream in a fixed order whatever the
 * outcomes, and the sphere a candidate is tried for is the next one still to be
 * placed. A batch of B candidates is therefore drawn at once; worker threads
 * test them, read-only, against the spheres placed before the batch, with the
 * largest radius any of them can be tried for (r_hi = max of the next B radii),
 * and keep for each candidate the spheres that overlap it at that radius (its
 * only possible conflicts with the old spheres: fl(r_i + r_q) <= fl(r_hi + r_q)),
 * with their squared distances. The main thread then takes the candidates in
 * order with the one-by-one rule: the exact test against that short list and
 * against the spheres placed earlier in the same batch. The placements, and the
 * count of rejected candidates, are those of the one-by-one process.
 *
 * The spheres are held in two grids: those up to r_cut (1.5 times the mean
 * radius) in a fine grid of cell side >= 2 r_cut, the larger ones in a coarse
 * grid of cell side >= 2 r_max, so that a wide size distribution does not make
 * every search walk the long cell lists of a grid sized by its largest sphere. A
 * search for radius R visits the fine cells within R + r_cut and the coarse cells
 * within R + r_max of the candidate; which spheres are visited does not change
 * the outcome of the exact test. */
enum { kBatch = 8192, kList = 6 };

typedef struct {
  double c[3];
  double d2[kList], rq[kList];  /* squared minimum-image distance and radius of each possible conflict */
  int nq;                       /* kList + 1: more than kList conflicts, test against all old spheres */
} rsa_cand;

typedef struct {
  int64_t ng;     /* cells per side */
  double r_in;    /* the largest radius held (r_cut or r_max) */
  int64_t* head;  /* first sphere of each cell, -1 when empty */
  uint64_t* touched; /* cells that received a sphere in the current batch */
} rsa_grid;

typedef struct {
  rsa_grid g[2];  /* fine, coarse */
  int ngrid;
  const rsa_node* node;
  rsa_cand* cand;
  int64_t ncand;
  double r_hi;
  int nthreads;
} rsa_pool;

typedef struct {
  rsa_pool* pool;
  int tid;
} rsa_worker_arg;

static double dist2(double px, double py, double pz, const rsa_node* q) {
  const double ddx = minimg(px - q->x), ddy = minimg(py - q->y), ddz = minimg(pz - q->z);
  return ddx * ddx + ddy * ddy + ddz * ddz;
}

static int overlaps(double px, double py, double pz, double ri, const rsa_node* q) {
  const double rr = ri + q->r;
  return dist2(px, py, pz, q) <= rr * rr;
}

/* Cells of grid g to visit around p for a search radius R: offsets -s..s per axis
 * (every cell once when 2 s + 1 covers the axis). Two points closer than D along an
 * axis lie in cells at most floor(D ng) + 1 apart; the 1e-12 covers the rounding of
 * the products x ng that place them in cells. */
typedef struct {
  int64_t lo, cnt, c0[3];
} rsa_span;

static rsa_span grid_span(const rsa_grid* g, double px, double py, double pz, double R) {
  rsa_span sp;
  const int64_t ng = g->ng;
  int64_t s = (int64_t)floor((R + g->r_in) * (double)ng + 1e-12) + 1;
  if (2 * s + 1 >= ng) {
    sp.lo = 0;
    sp.cnt = ng;
    sp.c0[0] = sp.c0[1] = sp.c0[2] = -1; /* absolute cells 0 .. ng - 1 */
  } else {
    sp.lo = -s;
    sp.cnt = 2 * s + 1;
    sp.c0[0] = cell_index(px, ng);
    sp.c0[1] = cell_index(py, ng);
    sp.c0[2] = cell_index(pz, ng);
  }
  return sp;
}

static int64_t span_cell(const rsa_grid* g, const rsa_span* sp, int64_t oz, int64_t oy, int64_t ox) {
  const int64_t ng = g->ng;
  int64_t a[3];
  const int64_t o[3] = {ox, oy, oz};
  for (int d = 0; d < 3; ++d) {
    if (sp->c0[d] < 0) {
      a[d] = o[d];
    } else {
      /* |lo + o| <= s < ng / 2: one wrap at most */
      const int64_t v = sp->c0[d] + sp->lo + o[d];
      a[d] = v < 0 ? v + ng : (v >= ng ? v - ng : v);
    }
  }
  return (a[2] * ng + a[1]) * ng + a[0];
}

static void conflicts(const rsa_pool* P, rsa_cand* k) {
  const double px = k->c[0], py = k->c[1], pz = k->c[2];
  k->nq = 0;
  for (int gi = 0; gi < P->ngrid; ++gi) {
    const rsa_grid* g = &P->g[gi];
    const rsa_span sp = grid_span(g, px, py, pz, P->r_hi);
    for (int64_t oz = 0; oz < sp.cnt; ++oz)
      for (int64_t oy = 0; oy < sp.cnt; ++oy)
        for (int64_t ox = 0; ox < sp.cnt; ++ox) {
          const int64_t cell = span_cell(g, &sp, oz, oy, ox);
          for (int64_t j = g->head[cell]; j >= 0; j = P->node[j].next) {
            const rsa_node* q = &P->node[j];
            const double d2 = dist2(px, py, pz, q), rr = P->r_hi + q->r;
            if (d2 <= rr * rr) {
              if (k->nq == kList) {
                k->nq = kList + 1;
                return;
              }
              k->d2[k->nq] = d2;
              k->rq[k->nq++] = q->r;
            }
          }
        }
  }
}

/* Conflict lists of the candidates k = tid, tid + nthreads, ... of the batch. */
static void* rsa_worker(void* p) {
  rsa_worker_arg* a = (rsa_worker_arg*)p;
  const rsa_pool* P = a->pool;
  for (int64_t k = a->tid; k < P->ncand; k += P->nthreads) conflicts(P, &P->cand[k]);
  return NULL;
}

/* Exact one-by-one test of candidate k for radius ri: its conflict list (or all
 * old spheres when the list overflowed) and the spheres placed since the batch
 * began (indices >= first_new, at the heads of the lists of the touched cells). */
static int accepted(const rsa_pool* P, const rsa_cand* k, double ri, int64_t first_new) {
  const double px = k->c[0], py = k->c[1], pz = k->c[2];
  const int listed = k->nq <= kList;
  if (listed) {
    for (int t = 0; t < k->nq; ++t) {
      const double rr = ri + k->rq[t];
      if (k->d2[t] <= rr * rr) return 0;
    }
  }
  for (int gi = 0; gi < P->ngrid; ++gi) {
    const rsa_grid* g = &P->g[gi];
    const rsa_span sp = grid_span(g, px, py, pz, ri);
    for (int64_t oz = 0; oz < sp.cnt; ++oz)
      for (int64_t oy = 0; oy < sp.cnt; ++oy)
        for (int64_t ox = 0; ox < sp.cnt; ++ox) {
          const int64_t cell = span_cell(g, &sp, oz, oy, ox);
          if (listed && !((g->touched[cell >> 6] >> (cell & 63)) & 1u)) continue;
          for (int64_t j = g->head[cell]; j >= 0; j = P->node[j].next) {
            if (j < first_new && listed) break; /* the old spheres were covered by the list */
            if (overlaps(px, py, pz, ri, &P->node[j])) return 0;
          }
        }
  }
  return 1;
}

static int grid_init(rsa_grid* g, double r_in) {
  int64_t ng = (int64_t)floor(1.0 / (2.0 * r_in * (1.0 + 1e-9)));
  if (ng < 1) ng = 1;
  while (ng > 1 && ng * ng * ng > ((int64_t)1 << 28)) --ng;
  const int64_t ncell = ng * ng * ng;
  g->ng = ng;
  g->r_in = r_in;
  g->head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
  g->touched = (uint64_t*)calloc((size_t)((ncell + 63) / 64), sizeof(uint64_t));
  if (!g->head || !g->touched) return 0;
  for (int64_t c = 0; c < ncell; ++c) g->head[c] = -1;
  return 1;
}

static int rsa_batched(int64_t n, uint64_t seed, const double* r, double* x, int64_t max_reject, int64_t* rejects_out,
                       int nthreads) {
  double rmax = 0.0, rsum = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(r[i] > 0.0) || r[i] >= 0.25) return 1;
    if (r[i] > rmax) rmax = r[i];
    rsum += r[i];
  }
  /* two grids only when a grid sized by the largest sphere would hold many spheres
     per cell; the fine cells hold at least the volume of one sphere per particle */
  double r_cut = 1.5 * rsum / (double)n;
  const double half_side = 0.5 * cbrt(1.0 / (double)n);
  if (r_cut < half_side) r_cut = half_side;
  const double coarse_cells = pow(floor(1.0 / (2.0 * rmax * (1.0 + 1e-9))), 3.0);
  if (r_cut > rmax || (double)n < 8.0 * coarse_cells) r_cut = rmax;
  rsa_pool P;
  memset(&P, 0, sizeof(P));
  P.ngrid = r_cut < rmax ? 2 : 1;
  rsa_node* node = (rsa_node*)malloc(sizeof(rsa_node) * (size_t)n);
  rsa_cand* cand = (rsa_cand*)malloc(sizeof(rsa_cand) * kBatch);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  rsa_worker_arg* wa = (rsa_worker_arg*)malloc(sizeof(rsa_worker_arg) * (size_t)nthreads);
  int64_t* placed = (int64_t*)malloc(sizeof(int64_t) * 2 * kBatch); /* (grid, cell) of the batch's spheres */
  int ok_alloc = node && cand && th && wa && placed && grid_init(&P.g[0], r_cut);
  if (ok_alloc && P.ngrid == 2) ok_alloc = grid_init(&P.g[1], rmax);
  if (!ok_alloc) {
    for (int gi = 0; gi < 2; ++gi) {
      free(P.g[gi].head);
      free(P.g[gi].touched);
    }
    free(node); free(cand); free(th); free(wa); free(placed);
    return 4;
  }
  P.node = node;
  P.cand = cand;
  P.nthreads = nthreads;
  int rc = 0;
  uint64_t s = stream_state(seed, 1);
  int64_t rejects = 0, i = 0;
  while (rc == 0 && i < n) {
    /* draw a batch; the radius bound covers every sphere it can be tried for */
    const int64_t nb = kBatch;
    double r_hi = 0.0;
    for (int64_t t = i; t < n && t < i + nb; ++t)
      if (r[t] > r_hi) r_hi = r[t];
    for (int64_t k = 0; k < nb; ++k) {
      cand[k].c[0] = u01(&s);
      cand[k].c[1] = u01(&s);
      cand[k].c[2] = u01(&s);
    }
    P.ncand = nb;
    P.r_hi = r_hi;
    /* the conflict lists, one slice per thread; a slice whose thread could not be
       started is done here */
    int ok[64];
    for (int t = 1; t < nthreads; ++t) {
      wa[t].pool = &P;
      wa[t].tid = t;
      ok[t] = pthread_create(&th[t], NULL, rsa_worker, &wa[t]) == 0;
    }
    wa[0].pool = &P;
    wa[0].tid = 0;
    rsa_worker(&wa[0]);
    for (int t = 1; t < nthreads; ++t) {
      if (ok[t])
        pthread_join(th[t], NULL);
      else
        rsa_worker(&wa[t]);
    }
    const int64_t first_new = i;
    int64_t nplaced = 0;
    for (int64_t k = 0; k < nb && i < n; ++k) {
      if (accepted(&P, &cand[k], r[i], first_new)) {
        const double px = cand[k].c[0], py = cand[k].c[1], pz = cand[k].c[2];
        x[i] = px; x[n + i] = py; x[2 * n + i] = pz;
        const int gi = (P.ngrid == 2 && r[i] > r_cut) ? 1 : 0;
        rsa_grid* g = &P.g[gi];
        const int64_t ng = g->ng;
        const int64_t c = (cell_index(pz, ng) * ng + cell_index(py, ng)) * ng + cell_index(px, ng);
        node[i].x = px;
        node[i].y = py;
        node[i].z = pz;
        node[i].r = r[i];
        node[i].next = g->head[c];
        g->head[c] = i;
        g->touched[c >> 6] |= (uint64_t)1 << (c & 63);
        placed[2 * nplaced] = gi;
        placed[2 * nplaced + 1] = c;
        ++nplaced;
        ++i;
      } else if (++rejects > max_reject) {
        rc = 3;
        break;
      }
    }
    for (int64_t t = 0; t < nplaced; ++t) P.g[placed[2 * t]].touched[placed[2 * t + 1] >> 6] = 0;
  }
  for (int gi = 0; gi < 2; ++gi) {
    free(P.g[gi].head);
    free(P.g[gi].touched);
  }
  free(node); free(cand); free(th); free(wa); free(placed);
  if (rejects_out) *rejects_out = rejects;
  return rc;
}

int pcgen_rsa(int64_t n, uint64_t seed, const double* r, double* x, int64_t max_reject, int64_t* rejects_out) {
  if (n < 0 || !r || !x) return 1;
  if (n == 0) return 0;
  long cores = sysconf(_SC_NPROCESSORS_ONLN);
  const char* env = getenv("PCGEN_THREADS");
  if (env && atoi(env) > 0) cores = atoi(env);
  const int nthreads = (int)(cores < 1 ? 1 : (cores > 64 ? 64 : cores));
  /* PCGEN_MIN_BATCHED lowers the size from which the batched placement runs (tests) */
  const char* mb = getenv("PCGEN_MIN_BATCHED");
  const int64_t min_batched = (mb && atoll(mb) > 0) ? atoll(mb) : ((int64_t)1 << 18);
  if (n < min_batched || nthreads < 2) return rsa_sequential(n, seed, r, x, max_reject, rejects_out);
  return rsa_batched(n, seed, r, x, max_reject, rejects_out, nthreads);
}

/* The one-by-one process, for tests of the batched placement. */
int pcgen_rsa_sequential(int64_t n, uint64_t seed, const double* r, double* x, int64_t max_reject,
                         int64_t* rejects_out) {
  return rsa_sequential(n, seed, r, x, max_reject, rejects_out);
}
