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
 * Build: cc -O2 -ffp-contract=off -fPIC -shared gen.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

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
int pcgen_rsa(int64_t n, uint64_t seed, const double* r, double* x, int64_t max_reject, int64_t* rejects_out) {
  if (n < 0 || !r || !x) return 1;
  if (n == 0) return 0;
  double rmax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(r[i] > 0.0) || r[i] >= 0.25) return 1;
    if (r[i] > rmax) rmax = r[i];
  }
  /* grid side >= 2*rmax, at most 2^21 cells per axis product bound */
  int64_t ng = (int64_t)floor(1.0 / (2.0 * rmax * (1.0 + 1e-9)));
  if (ng < 1) ng = 1;
  while (ng > 1 && ng * ng * ng > ((int64_t)1 << 30)) --ng;
  int64_t ncell = ng * ng * ng;
  int32_t* head = (int32_t*)malloc(sizeof(int32_t) * (size_t)ncell);
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!head || !next) { free(head); free(next); return 4; }
  for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
  uint64_t s = stream_state(seed, 1);
  int64_t rejects = 0;
  int span = ng >= 3 ? 1 : 0; /* ng < 3: every cell is a neighbour; scan all once */
  for (int64_t i = 0; i < n; ++i) {
    for (;;) {
      double px = u01(&s), py = u01(&s), pz = u01(&s);
      int64_t cx = (int64_t)(px * ng), cy = (int64_t)(py * ng), cz = (int64_t)(pz * ng);
      if (cx >= ng) cx = ng - 1;
      if (cy >= ng) cy = ng - 1;
      if (cz >= ng) cz = ng - 1;
      int ok = 1;
      int64_t lo = span ? -1 : 0, hi = span ? 1 : ng - 1;
      for (int64_t dz = lo; dz <= hi && ok; ++dz)
        for (int64_t dy = lo; dy <= hi && ok; ++dy)
          for (int64_t dx = lo; dx <= hi && ok; ++dx) {
            int64_t ax = span ? (cx + dx + ng) % ng : dx;
            int64_t ay = span ? (cy + dy + ng) % ng : dy;
            int64_t az = span ? (cz + dz + ng) % ng : dz;
            for (int32_t j = head[(az * ng + ay) * ng + ax]; j >= 0; j = next[j]) {
              double ddx = minimg(px - x[j]), ddy = minimg(py - x[n + j]), ddz = minimg(pz - x[2 * n + j]);
              double rr = r[i] + r[j];
              if (ddx * ddx + ddy * ddy + ddz * ddz <= rr * rr) { ok = 0; break; }
            }
          }
      if (ok) {
        x[i] = px; x[n + i] = py; x[2 * n + i] = pz;
        int64_t c = (cz * ng + cy) * ng + cx;
        next[i] = head[c];
        head[c] = (int32_t)i;
        break;
      }
      if (++rejects > max_reject) { free(head); free(next); if (rejects_out) *rejects_out = rejects; return 3; }
    }
  }
  free(head);
  free(next);
  if (rejects_out) *rejects_out = rejects;
  return 0;
}
