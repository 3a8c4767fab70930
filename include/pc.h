/*
 * pc — per-time-step particle operator of arXiv 2501.05340 on one GB300 (sm_103a).
 *
 *   collide: deterministic hard-sphere binary collisions (Sec. 2.4, 3.3, 4.3)
 *   project: Gaussian projection of particle sources onto the Legendre-Gauss
 *            nodes of hexahedral DG elements with discrete normalisation (Sec. 2.3, 4.2)
 *
 * C ABI: plain pointers and sizes, no C++ or torch types. All particle, source
 * and field buffers are DEVICE memory owned by the caller; the context owns its
 * scratch, sized once by pc_init (no allocation in pc_collide / pc_project).
 * Every call queues its work on the context's stream and returns without
 * waiting for the GPU, unless stated otherwise.
 *
 * Domain: the periodic unit cube [0,1)^3. Per-particle vectors are SoA: a
 * "[3][n]" array holds the n first coordinates, then the n second, then the n
 * third. Fields are field[elem][comp][k][j][i] with elem = (ez*ne + ey)*ne + ex
 * and i the fastest Gauss-node index; comp 0..2 momentum, 3 energy.
 *
 * Errors: every call returns a pc_status. Argument errors are detected before any
 * work is queued and leave all buffers untouched. Conditions found on the GPU
 * (matching did not converge, a candidate list overflowed) are recorded in the
 * context and reported by the next pc_get_stats / pc_sync, which wait for the
 * stream. pc_last_error gives a one-line message for the last failure.
 */
#ifndef PC_H
#define PC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PC_OK = 0,
  PC_EINVAL = 1,       /* invalid argument (null pointer, size, parameter out of range) */
  PC_ENOMEM = 2,       /* device allocation failed (pc_init only) */
  PC_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  PC_ENOCONVERGE = 4,  /* the matching rounds reached their cap (cannot happen for valid input) */
  PC_ECAPACITY = 5,    /* a capacity was exceeded (candidate partners per particle, fixed scratch) */
  PC_ETIMEOUT = 6,     /* a bounded wait inside a kernel expired (the kernel stopped cleanly) */
  PC_EREPLAY = 7,      /* a given pair has no contact within the step any more (replay / adjoint) */
} pc_status;

typedef struct pc_ctx pc_ctx;

/* Operator configuration, fixed for the lifetime of a context. */
typedef struct {
  int64_t n_max;        /* largest particle count a call will pass (> 0) */
  int32_t ne;           /* elements per side of the periodic unit cube (>= 3) */
  int32_t degree;       /* DG degree N: N+1 Legendre-Gauss nodes per axis, 0..15 */
  double sigma;         /* Gaussian kernel width (> 0) */
  double cutoff_sigmas; /* kernel cutoff radius in units of sigma (> 0); 3 in the paper's workloads */
  int32_t cutoff_kind;  /* 0: box |d_axis| <= cutoff on every axis (separable); 1: sphere |d| <= cutoff */
  double restitution;   /* normal restitution coefficient e in [0, 1] (Sec. 2.4) */
  double reach_hint;    /* expected largest reach 2 r_max + 2 v_max dt of a step; sizes the
                           collision cells (side >= reach_hint). 0 < reach_hint < 0.5.
                           A step whose actual reach exceeds the hint stays exact (more
                           cells are searched) as long as it stays below 0.5 box lengths,
                           where the periodic minimum image is the only image that can
                           collide; a step with a reach >= 0.5 is refused on the GPU
                           (PC_EINVAL from the next pc_sync, outputs undefined). */
  int32_t cand_cap;     /* candidate partners kept per particle and step (1..32; 0 = 16) */
  void* stream;         /* cudaStream_t for all work (NULL = legacy default stream) */
  double amp;           /* curved-mesh amplitude a of x = xi + a (sin 2pi xi_y sin 2pi xi_z, cyclic);
                           0 = affine. Used by pc_project_curved_f32 (needs cutoff_kind 1), 0 <= a < 0.04 */
} pc_config;

/* Device SoA particle state (FP64). */
typedef struct {
  int64_t n;     /* particle count, 0 <= n <= n_max */
  int32_t* id;   /* [n] unique ids; ties in contact time go to the smaller id */
  double* x;     /* [3][n] centres in [0,1) */
  double* v;     /* [3][n] velocities */
  double* r;     /* [n] radii (> 0) */
  double* m;     /* [n] masses (> 0) */
  double* q;     /* [4][n] sources (3 momentum + 1 energy), or NULL */
} pc_particles;

/* Device particle state of the mixed-precision path (FP32 storage).
 * Positions are cell-relative: cell[p] is the linear index (cz*nc + cy)*nc + cx of
 * the context's nc^3 collision grid (pc_cells_per_side) and o[a][p] in [0,1) the
 * FP32 offset inside that cell in cell units, so the position is (c_a + o_a)/nc. */
typedef struct {
  int64_t n;      /* particle count, 0 <= n <= n_max */
  int32_t* id;    /* [n] unique ids */
  int32_t* cell;  /* [n] linear collision cell */
  float* o;       /* [3][n] offsets in cell units, [0,1) */
  float* v;       /* [3][n] velocities */
  float* r;       /* [n] radii (> 0) */
  float* m;       /* [n] masses (> 0) */
  float* q;       /* [4][n] sources, or NULL */
} pc_particles_f32;

/* Tensor-core operand type of pc_project_f32. */
typedef enum { PC_TC_F16 = 0, PC_TC_BF16 = 1 } pc_tc_type;

typedef struct {
  int64_t pairs;          /* collisions committed in the last pc_collide */
  int64_t candidates;     /* candidate pairs (finite contact time) counted from both ends */
  int64_t worklist;       /* particles left after the first matching round */
  int64_t rounds;         /* matching rounds in the last pc_collide (>= 1 when pairs > 0) */
  int64_t fp64_solves;    /* exact FP64 contact solves after the FP32 reject filter */
  int64_t max_candidates; /* largest per-particle candidate count */
  int32_t cells_per_side; /* collision cells per side */
  int32_t stencil;        /* neighbour cells searched on each side in the last step */
  int32_t device_status;  /* pc_status recorded on the GPU (PC_OK when clean) */
  int64_t kernel_launches; /* kernels this context has launched since pc_init */
} pc_stats;

/* Phases timed by pc_set_timing / pc_get_timing. */
typedef enum {
  PC_PH_BIN = 0,     /* collide: cell keys, scan, scatter, per-cell order */
  PC_PH_GATHER = 1,  /* collide: sorted copies of the state */
  PC_PH_SEARCH = 2,  /* collide: contact search */
  PC_PH_MATCH = 3,   /* collide: matching rounds */
  PC_PH_RESPOND = 4, /* collide: response, advance, output state */
  PC_PH_PBIN = 5,    /* project: element keys, scan, scatter, per-element order */
  PC_PH_FACTORS = 6, /* project: normalised 1-D kernel factors */
  PC_PH_DEPOSIT = 7, /* project: per-element gather of the deposit */
  PC_NPHASE = 8
} pc_phase;

/* Pair selection of pc_collide / pc_collide_rot (Sec. 4.3: at most one collision per
 * particle per step). PC_PAIRS_EARLIEST (the default): earliest contact first, ties
 * to the smaller id pair. PC_PAIRS_SFC_FIRST: the paper's first-found order, with the
 * particles visited along a space-filling curve and each free particle taking the
 * first free partner of a valid collision in that order; the curve is the Morton
 * (Z-order) curve over the collision cells (bit b of the cell's x, y, z index to bit
 * 3b, 3b+1, 3b+2), particles within a cell by id, so the result depends on the cell
 * grid (pc_cells_per_side). Either matching is computed in parallel and is unique. */
typedef enum { PC_PAIRS_EARLIEST = 0, PC_PAIRS_SFC_FIRST = 1 } pc_pair_policy;
pc_status pc_set_pair_policy(pc_ctx* ctx, int32_t policy);

/* Create a context: validates cfg, builds the Gauss tables, chooses the collision
 * cells (side >= reach_hint, at least 3 per side) and allocates all scratch on
 * the current CUDA device. *ctx is NULL on failure. */
pc_status pc_init(pc_ctx** ctx, const pc_config* cfg);

/* One collision step of length dt (Sec. 3.3, 4.3). Reads `in` in any order and
 * writes `out` (distinct buffers, same n; `out->q` may be NULL only if `in->q` is):
 * particles sorted by collision cell of their start-of-step position (ties by id),
 * advanced by dt. Candidate pairs: both roots of |dx + t dv| = r_i + r_j positive,
 * approaching, smaller root t <= dt, dx the periodic minimum image. Each particle
 * collides at most once per step; pairs are chosen earliest-contact-first with
 * ties to the smaller id pair, which is the greedy matching in the order
 * (t, min id, max id). Response: frictionless impulse J = -m_r (1+e) v_r.n, then
 * x' = x + t v + (dt - t) v'; free particles x' = x + dt v; then x' wrapped into
 * [0,1). FP64 arithmetic in a fixed operation order without fused multiply-add,
 * so pairs, times, x' and v' are bit-identical to a plain IEEE implementation. */
pc_status pc_collide(pc_ctx* ctx, const pc_particles* in, pc_particles* out, double dt);

/* One collision step with Coulomb friction and rotation (Sec. 2.4 jump relations of
 * linear and angular momentum): the pairs of pc_collide (they do not depend on the
 * spin), then for each pair, from each particle's own side (it is particle 1, n from
 * it to its partner): J = J_n n + J_t t, J_n = -m_r (1+e) v_r.n; contact-point
 * velocity v_c = v_r + r_1 w_1 x n + r_2 w_2 x n (the two rotational terms added
 * lower id first); v_rt = v_c - (v_c.n) n; J_t = max(mu J_n, -(2/7)(1+e) m_r |v_rt|)
 * (sliding, else sticking), t = v_rt / |v_rt| (no tangential impulse when |v_rt| =
 * 0); v' = v + J/m, w' = w + r (n x J) / I with I = (2/5) m r^2 (solid spheres);
 * x' = x + t v + (dt - t) v'. w_in: device angular velocities [3][n] in the order of
 * `in`; w_out: [3][n] in the order of `out` (cell-sorted like the other outputs);
 * distinct buffers. mu >= 0 (mu = 0 leaves w unchanged and gives pc_collide's
 * velocities). FP64 in a fixed operation order without fused multiply-add: bit-
 * identical to the plain IEEE implementation. Other arguments as pc_collide. */
pc_status pc_collide_rot(pc_ctx* ctx, const pc_particles* in, pc_particles* out, const double* w_in, double* w_out,
                         double mu, double dt);

/* Projection (Sec. 2.3, 4.2 with a Gaussian shape function): for every Gauss node
 * X_g, field[g][c] = sum_p q[c][p] K(X_g - x_p) / Z_p, Z_p = sum_g W_g K(X_g - x_p),
 * W_g = w_i w_j w_k (h/2)^3, K(d) = exp(-|d|^2/(2 sigma^2)) inside the cutoff and 0
 * outside, d the periodic minimum image. Hence sum_g W_g field[g][c] = sum_p q[c][p].
 * p->q must be non-NULL. field: device [ne^3][4][(N+1)^3] doubles, overwritten.
 * Accuracy: within 1e-12 of the exact sum, normwise per component. */
pc_status pc_project(pc_ctx* ctx, const pc_particles* p, double* field);

/* Linear corner-node deposition (Sec. 2.3: the continuous, linear variant of inverse
 * distance weighting, each source spread over the 8 vertices of the element that
 * contains it; Sec. 4.2: corner nodes with
 * unique periodic ids, deposition radius one element) on the affine mesh. A
 * particle at reference position xi in [-1,1]^3 of its element (xi_a = 2 (x_a ne -
 * e_a) - 1) gives q[c][p] w_d(xi) to corner d of the element, w_d(xi) =
 * prod_a (1 -/+ xi_a)/2 for the lower / upper corner along axis a. Node n holds the
 * density S_n / V_n, S_n its sum over all particles, V_n = the sum over the 8
 * elements around it of sum_g W_g w_n(xi_g) (= h^3 here). The field at the Gauss
 * nodes of an element is the trilinear interpolation of its 8 corner densities, so
 * sum_g W_g field[g][c] = sum_p q[c][p]. p->q must be non-NULL; positions in
 * [0,1)^3 (else PC_EINVAL from pc_sync). field: device [ne^3][4][(N+1)^3] doubles,
 * overwritten. FP64-accurate (double-float sums and products, one FP64 FMA per
 * output), deterministic (particles summed by element, then id). Sources are
 * taken to 46 significant bits; magnitudes below 2^-126 count as zero, from
 * 2^128 on as infinite. Accuracy: within 1e-12 of the exact sums, normwise per
 * component. */
pc_status pc_project_idw(pc_ctx* ctx, const pc_particles* p, double* field);

/* Nearest-DOF (Dirac delta) deposition (Sec. 4.2): the whole source of a particle
 * goes to the Gauss node of its element nearest to it, which is the per-axis nearest
 * node in reference coordinates (the lower index on an exact tie), as the density
 * q[c][p] / W_g, W_g = w_i w_j w_k (h/2)^3; the nearest node of the own element is
 * also the nearest of the whole mesh. Arguments and layout as pc_project_idw. FP64,
 * deterministic; a particle within rounding of a midpoint between two nodes may
 * choose either. */
pc_status pc_project_dirac(pc_ctx* ctx, const pc_particles* p, double* field);

/* Field evaluation at the particles (Sec. 3.2): out[c][p] = sum_{ijk} field[e][c][k][j][i]
 * l_i(xi_1) l_j(xi_2) l_k(xi_3) for the particle's element e and reference position
 * xi_a = 2 (x_a ne - e_a) - 1, l the Lagrange basis of the Legendre-Gauss nodes (the
 * DG polynomial of the field). field: device [ne^3][nvar][(N+1)^3] doubles; out:
 * device [nvar][n] in the order of p; 1 <= nvar <= 16; positions in [0,1)^3 (else
 * PC_EINVAL from pc_sync). FP64-accurate (double-float sums and products; the
 * reference coordinate to 2^-47): within 1e-12 of the exact value normwise per
 * variable for N <= 7; for higher N the coordinate's error, amplified by the basis'
 * derivative (~(N+1)^2), allows up to ~2e-11. Deterministic. */
pc_status pc_eval_field(pc_ctx* ctx, const pc_particles* p, const double* field, int32_t nvar, double* out);

/* Drag-force sources (Sec. 2.2 particle momentum equation, Sec. 2.3 source terms):
 * F = 3 pi mu_f d f_D (u_f - v_p) with d = 2 r, f_D = 1 + 0.15 Re^0.687 (Schiller-
 * Naumann; the paper's correlation is not printed) and Re = rho_f |u_f - v_p| d / mu_f;
 * q[4][n] = (-F, -F.v_p), the per-particle sources whose projection is the fluid's
 * momentum and energy source. fluid: device [4][n] = (rho_f, u_f) at the particles (for
 * example pc_eval_field of a 4-variable field), in the order of p; q may be p->q. FP64. */
pc_status pc_drag_sources(pc_ctx* ctx, const pc_particles* p, const double* fluid, double mu_f, double* q);

/* ---- differentiation (no counterpart in the paper) ----
 * The gradient of a rollout is taken with each step's pair set held fixed. The
 * calls below work on particle arrays in one fixed order (for example by id), not
 * on the cell-sorted order that pc_collide writes. */

/* Scatter the pairs of the last pc_collide into partner[id] (device, n_ids
 * entries): the partner's id, or -1. Ids must lie in [0, n_ids). */
pc_status pc_pairs_to_partner(pc_ctx* ctx, int32_t* partner, int64_t n_ids);

/* One step with a given pair set (partner[p] = index of p's partner in the same
 * arrays, or -1): contact times from the formula of pc_collide, the same response
 * and advance, no search and no reordering; `out` in the order of `in` (r, m, id,
 * q copied when out's pointers differ from in's). Bit-identical to pc_collide for
 * the pair set pc_collide chose. A pair without a root in [0, dt] is recorded as
 * PC_EREPLAY (reported by pc_sync). */
pc_status pc_collide_replay(pc_ctx* ctx, const pc_particles* in, pc_particles* out, const int32_t* partner,
                            double dt);

/* Vector-Jacobian product of pc_collide_replay at the pre-step state `in`: given
 * device cotangents gx_out, gv_out [3][n] of the new positions and velocities,
 * writes gx_in, gv_in [3][n] of the old ones. The contact time is differentiated
 * through |dx + t dv| = r_i + r_j (implicit function theorem), the wrap has
 * derivative 1. */
pc_status pc_collide_adjoint(pc_ctx* ctx, const pc_particles* in, const int32_t* partner, double dt,
                             const double* gx_out, const double* gv_out, double* gx_in, double* gv_in);

/* Vector-Jacobian product of pc_project: given G = dL/dfield (device, field
 * layout), writes gq[4][n] = dL/dq and gx[3][n] = dL/dx (the Gaussian and the
 * normalisation Z_p differentiated, the cutoff held fixed), in the order of p. FP64. */
pc_status pc_project_adjoint(pc_ctx* ctx, const pc_particles* p, const double* G, double* gq, double* gx);

/* ---- mixed-precision path ---- */

/* Collision cells per side of the context's grid (the nc of pc_particles_f32). */
int32_t pc_cells_per_side(const pc_ctx* ctx);

/* Convert an FP64 state to the FP32 cell-relative storage, same order:
 * s = x nc (FP64), c = floor(s) clamped to [0, nc), o = float(s - c); an offset
 * that rounds to 1 is carried into the next cell (periodically). v, r, m, q are
 * rounded to FP32. out->q may be NULL. Device buffers; queued on the stream. */
pc_status pc_quantize(pc_ctx* ctx, const pc_particles* in, pc_particles_f32* out);

/* One collision step on the FP32 cell-relative storage (`in` -> `out`, distinct,
 * out sorted by cell, ties by id). Same pair selection as pc_collide, on the exact
 * FP64 values of the stored state in cell units: x = c + o, v nc, (r_i + r_j) nc,
 * periodic box of nc cells. A certified FP32 filter on cell-relative differences
 * rejects pairs before the FP64 solve. Colliding pairs: FP64 response (as
 * pc_collide, positions in cell units), new position stored as cell + FP32
 * offset, velocity rounded to FP32. Free particles: o' = o + float(dt nc) v in
 * FP32 with a carry into the neighbouring cell, so a step needs |v_a| dt nc < 1 on
 * every axis (the cells' side >= reach_hint >= 2 v_max dt gives it whenever the hint
 * bounds the step's reach; a larger move leaves an offset outside [0, 1), which the
 * next step reports as PC_EINVAL). Bit-identical to a plain implementation of these
 * rules. */
pc_status pc_collide_f32(pc_ctx* ctx, const pc_particles_f32* in, pc_particles_f32* out, double dt);

/* One mixed step with a given pair set (partner[p] = index of p's partner in the
 * same arrays, or -1), in the order of `in`: the contact time of pc_collide_f32's
 * search (FP64, cell units, from p's side), then the same free flight and response
 * (arXiv 2501.05340 Sec. 2.4 with the stored-state rules of pc_collide_f32), so
 * bit-identical to pc_collide_f32 for the pair set it chose. out's cell, o and v
 * must be distinct from in's; r, m, id, q are copied when out's pointers differ
 * from in's. A pair without a root in [0, dt] is recorded as PC_EREPLAY and both
 * particles fly free. Not in the paper: the forward pass of FP32 rollouts. */
pc_status pc_collide_replay_f32(pc_ctx* ctx, const pc_particles_f32* in, pc_particles_f32* out, const int32_t* partner,
                                double dt);

/* Vector-Jacobian product of pc_collide_replay_f32 at the pre-step state `in`, in
 * FP32 and physical units (x = (cell + o) / nc): given device cotangents gx_out,
 * gv_out [3][n] of the new positions and velocities, writes gx_in, gv_in [3][n]
 * (distinct buffers) of the old ones. The storage rounding is taken as the
 * identity; the contact time is the forward step's FP64 root, differentiated
 * through |dx + t dv| = r_i + r_j in FP32. Not in the paper. */
pc_status pc_collide_adjoint_f32(pc_ctx* ctx, const pc_particles_f32* in, const int32_t* partner, double dt,
                                 const float* gx_out, const float* gv_out, float* gx_in, float* gv_in);

/* Vector-Jacobian product of pc_project_f32 in FP32 (box cutoff): given
 * G = dL/dfield (device FP32, field layout [ne^3][4][n1^3]), writes gq[4][n] =
 * dL/dq and gx[3][n] = dL/dx (physical units) in the order of p, with the inside-
 * cutoff decisions of the forward pass held fixed. Not in the paper. */
pc_status pc_project_adjoint_f32(pc_ctx* ctx, const pc_particles_f32* p, const float* G, float* gq, float* gx);

/* Projection of p->q (as pc_project) on the tensor cores: per element the
 * separable deposit is the dense contraction D[jk][c i] = sum_p (ky_j kz_k)(q_c kx_i),
 * each factor split into high and low parts of tc_type (FP16 or BF16), the three
 * significant products accumulated in FP32 (tcgen05, accumulators in tensor
 * memory). Kernel factors in FP32; cutoff decisions near the cutoff are made in
 * FP64 on the stored position, as in pc_project. field: device FP32
 * [ne^3][4][(N+1)^3], overwritten. Requires N + 1 <= 8 and (2 rho + 1)(N + 1) <= 32,
 * rho = ceil(cutoff_sigmas sigma ne).
 * Operand range (PC_TC_F16): the split operands are q_c k_x 2^4 / Z_x and
 * k_y k_z 2^8 / (Z_y Z_z), k <= 1, Z_a about 2 sqrt(2 pi) sigma ne. They overflow FP16
 * (65504) for |q| above about 4000 Z_x, and below 2^-3 the low half of the split is
 * subnormal, so the split's error becomes 2^-25 absolute (1e-5 relative near 3e-3).
 * Sources of order one sit far from both ends; scale others by a power of two (exact,
 * undone on the field) or use PC_TC_BF16, which has the exponent range of FP32. */
pc_status pc_project_f32(pc_ctx* ctx, const pc_particles_f32* p, float* field, int32_t tc_type);

/* Projection on the curved periodic mesh x = Phi(xi) = xi + amp (sin 2pi xi_y sin 2pi xi_z,
 * sin 2pi xi_z sin 2pi xi_x, sin 2pi xi_x sin 2pi xi_y) with the non-separable
 * physical-space Gaussian and a spherical cutoff (cfg.cutoff_kind = 1):
 * field[g][c] = sum_p q[c][p] K(X_g - x_p) / Z_p, X_g = Phi(xi_g) at the Gauss nodes,
 * Z_p = sum_g W_g K(X_g - x_p), W_g = w_i w_j w_k (h/2)^3 det DPhi(xi_g). Particles are
 * located in logical space by Newton's method on Phi(xi) = x (Sec. 3.2,
 * localisation). FP32 factors and accumulation; distances from double-float
 * positions; cutoff decisions with the squared distance within 2e-4 relative of the
 * squared cutoff made in FP64.
 * field: device FP32 [ne^3][4][(N+1)^3], overwritten. Deterministic (gather per
 * element). Requires cfg.amp > 0 or = 0, 2 pi sqrt(3) amp < 0.5. */
pc_status pc_project_curved_f32(pc_ctx* ctx, const pc_particles_f32* p, float* field);

/* Copy the pairs of the last pc_collide to HOST memory: ids[2k], ids[2k+1] (smaller
 * id first) and t[k], sorted by the smaller id. Writes min(cap, count) pairs and
 * the count to *npairs. Waits for the stream. PC_ECAPACITY if the device pair count
 * exceeds the pair buffers (n_max / 2 + 1; only after an earlier failed step). */
pc_status pc_get_pairs(pc_ctx* ctx, int32_t* ids, double* t, int64_t cap, int64_t* npairs);

/* Counters of the last pc_collide into HOST memory; returns the device status.
 * Waits for the stream. */
pc_status pc_get_stats(pc_ctx* ctx, pc_stats* out);

/* Wait for the stream; returns PC_ECUDA on an asynchronous CUDA error, else the
 * device status recorded since the last pc_sync (and clears it). */
pc_status pc_sync(pc_ctx* ctx);

/* Per-phase GPU timers, the counterpart of the per-stage timers of Sec. 4.4. While
 * on, every phase of pc_collide / pc_project records a pair of CUDA events on the
 * context's stream (no synchronisation). Off by default. */
pc_status pc_set_timing(pc_ctx* ctx, int on);

/* HOST outputs: ms[PC_NPHASE] summed phase durations and count[PC_NPHASE] recorded
 * phase instances since the previous call (either may be NULL); clears the records.
 * Records beyond 4096 phase instances between two calls are dropped (count stops).
 * Waits for the stream. */
pc_status pc_get_timing(pc_ctx* ctx, double* ms, int64_t* count);

/* Size in bytes of the fixed device array used by pc_project_noalloc. */
#define PC_NOALLOC_SCRATCH_BYTES (32u << 20)

/* The projection of pc_project for callers that may not allocate device memory:
 * for instance a plugin inside a host solver whose memory manager owns all of
 * the GPU's memory and forbids allocations by anyone else, or a time-critical
 * loop that cannot afford an allocation's latency or failure. There is no
 * counterpart in the paper; it computes exactly what pc_project computes.
 *
 * It needs no context and allocates nothing: no cudaMalloc, cudaFree or
 * allocating library call. Its scratch is one fixed device array of
 * PC_NOALLOC_SCRATCH_BYTES (32 MiB) compiled into the library, which every GPU
 * that loads the library holds until the process exits. The caller passes the
 * inputs (p: device SoA, p->q required) and the output (field: device
 * [ne^3][4][(N+1)^3] doubles, overwritten); cfg supplies ne, degree, sigma,
 * cutoff_sigmas, cutoff_kind (0) and stream; the other fields are ignored.
 * About 16 + 24 (2 rho + 1)(N+1) + 64 bytes per particle plus 8 ne^3 bytes must
 * fit in the array (rho = ceil(cutoff_sigmas sigma ne)); larger problems return
 * PC_ECAPACITY with the required size in msg.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture. The address is kept per device together with the id of
 * the context it belongs to; after a cudaDeviceReset the next call finds a new
 * context and looks the address up again (so, again, before any capture). The work is queued on cfg->stream and the call returns
 * without waiting; checks made on the GPU (positions outside [0,1)) are not
 * reported. All calls share the one array, which keeps the previous call's
 * contents (what must start at zero is cleared by each call): calls that overlap
 * on the GPU, on any streams, race and give wrong results. msg (optional, may be
 * NULL) receives a one-line message of at most msg_len - 1 characters. */
pc_status pc_project_noalloc(const pc_config* cfg, const pc_particles* p, double* field, char* msg,
                             int64_t msg_len);

/* Message of the last failure on this context (static storage of the context). */
const char* pc_last_error(const pc_ctx* ctx);

/* Release all scratch. Waits for the stream. NULL is accepted. */
void pc_destroy(pc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PC_H */
