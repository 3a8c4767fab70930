/*
 * CPU oracle for the particle collision and projection operator of
 * arXiv 2501.05340 (Schwarz, Kopper, de Staercke, Beck).
 *
 * TEST INFRASTRUCTURE ONLY. Plain, slow, FP64 C code that states what the GPU
 * path must compute. Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it. It shares no code with the CUDA library.
 *
 * Layouts: per-particle vectors are SoA, x[3][n] means x[0..n) are the first
 * coordinates, x[n..2n) the second, x[2n..3n) the third. The domain is the
 * periodic unit cube [0,1)^3. Fields are field[elem][comp][k][j][i] with
 * elem = (ez*ne + ey)*ne + ex and i the fastest node index.
 */
#ifndef PC_ORACLE_H
#define PC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Legendre-Gauss nodes eta[0..n1) (ascending) and weights w[0..n1) on [-1,1]
 * (Sec. 3.1: (N+1)^3 Legendre-Gauss points per element). Returns 0 on success. */
int or_gauss_legendre(int n1, double* eta, double* w);

/* Contact time of one pair (Sec. 3.3, Eq. collision-detect): the smaller root of
 * |dx + t dv| = r_i + r_j with dx = minimg(x_i - x_j), dv = v_i - v_j, if both
 * roots are positive, the particles approach, and the root is <= dt.
 * Returns the root, or +infinity when the pair is not a candidate. */
double or_contact_time(const double xi[3], const double xj[3], const double vi[3], const double vj[3],
                       double ri, double rj, double dt);

/* All candidate pairs (i<j, input index) by testing every pair. Writes at most
 * cap entries; returns the number of candidates found (may exceed cap). */
int64_t or_candidates_bruteforce(int64_t n, const double* x, const double* v, const double* r, double dt,
                                 int64_t cap, int64_t* ci, int64_t* cj, double* ct);

/* Same set via a cell list whose side is at least the largest possible reach
 * 2 r_max + 2 v_max dt (the halo criterion of Sec. 4.3). Falls back to the
 * brute force when fewer than 3 cells fit per side. */
int64_t or_candidates_cells(int64_t n, const double* x, const double* v, const double* r, double dt,
                            int64_t cap, int64_t* ci, int64_t* cj, double* ct);

/* One collision per particle (Sec. 4.3): global greedy matching of the
 * candidates in the strict order (t, min id, max id). partner[i] = index of the
 * partner or -1, tc[i] = contact time or +inf. Returns the number of pairs. */
int64_t or_match_greedy(int64_t n, const int32_t* id, int64_t ncand, const int64_t* ci, const int64_t* cj,
                        const double* ct, int64_t* partner, double* tc);

/* Same matching by rounds: every free particle picks its earliest free candidate
 * (ties to the smaller partner id); mutually-picked pairs are committed; repeat
 * until no free particle has a free candidate. *rounds receives the number of
 * rounds that committed at least one pair. Returns the number of pairs. */
int64_t or_match_rounds(int64_t n, const int32_t* id, int64_t ncand, const int64_t* ci, const int64_t* cj,
                        const double* ct, int64_t* partner, double* tc, int64_t* rounds);

/* Hard-sphere response of one committed pair (Sec. 2.4 jump relations, Sec. 3.3
 * velocity and position update) and free flight of everything else, then
 * periodic wrap. Arrays are updated in place. */
void or_respond_advance(int64_t n, double* x, double* v, const double* m, const int64_t* partner,
                        const double* tc, double e, double dt);

/* Response with Coulomb friction and rotation (Sec. 2.4): the jump relations of
 * linear and angular momentum with J = J_n n + J_t t, J_t = max(mu J_n,
 * -(2/7)(1+e) m_r |v_rt|) from the tangential contact-point velocity v_rt; moment
 * of inertia (2/5) m r^2. w[3][n] angular velocities, updated in place with x, v. */
void or_respond_advance_rot(int64_t n, double* x, double* v, double* w, const double* r, const double* m,
                            const int32_t* id, const int64_t* partner, const double* tc, double e, double mu,
                            double dt);

/* One whole collision step: candidates, greedy matching, response, advance.
 * partner/tc (length n) receive the matching. method: 0 cell list, 1 brute
 * force. Returns the number of pairs, or -1 on allocation failure. */
int64_t or_collide_step(int64_t n, double* x, double* v, const double* r, const double* m, const int32_t* id,
                        double e, double dt, int method, int64_t* partner, double* tc);

/* One collision step with the paper's first-found pair selection (Sec. 4.3: the
 * particles are visited in the order of the space-filling curve, each free particle
 * checks its possible partners in that order and the first valid collision with a
 * free partner is committed at once). Reading: the curve is the Morton (Z-order)
 * curve over the uniform grid of ncell^3 collision cells (bit b of the cell's x, y, z
 * index to bit 3b, 3b+1, 3b+2), particles within a cell by id; the candidates are
 * those of or_candidates_cells. Then or_respond_advance. Returns the number of
 * pairs, or -1 on allocation failure. */
int64_t or_collide_step_sfc(int64_t n, double* x, double* v, const double* r, const double* m, const int32_t* id,
                            double e, double dt, int64_t ncell, int64_t* partner, double* tc);

/* ---- mixed-precision storage (FP32 cell-relative state) ----
 * A position is stored as an integer cell c in [0, nc) per axis (linear cell
 * (cz*nc + cy)*nc + cx) and an FP32 offset o in [0,1) in cell units; velocities,
 * radii and masses as FP32. One step of the mixed method, read from the paper's
 * operator with this storage:
 *   contact detection: the a-priori test and root of or_contact_time on exact
 *     FP64 cell-unit values x = c + o, v = v_f nc, R = (r_i + r_j) nc, periodic
 *     box of nc cells;
 *   colliding pairs: the response of or_respond_advance in FP64 (velocities in
 *     physical units, positions in cell units), the new position wrapped into
 *     [0, nc), then stored as floor and FP32 offset, the velocity as FP32;
 *   free particles: o' = o + (dt nc)_f v_f in FP32, carried into the next or
 *     previous cell when o' leaves [0,1).
 * Arrays are updated in place. Returns the number of pairs (-1 on allocation
 * failure); partner/tc as in or_collide_step. */
int64_t or_collide_step_cellrel(int64_t n, int32_t nc, int32_t* cell, float* o, float* v, const float* r,
                                const float* m, const int32_t* id, double e, double dt, int64_t* partner,
                                double* tc);

/* ---- adjoint (not in the paper; gradients of the operator with the pair set held fixed) ----
 * Replay: one step with a given matching (partner[i] = index or -1), contact times
 * recomputed by or_contact_time's formula; returns -1 if a given pair has no root
 * in [0, dt] any more. x, v updated in place as or_respond_advance. */
int or_collide_replay(int64_t n, double* x, double* v, const double* r, const double* m, const int64_t* partner,
                      double e, double dt);

/* Vector-Jacobian product of one replayed step: given the cotangents gx_out, gv_out
 * of the new state, returns gx_in, gv_in of the pre-step state (x, v). The
 * contact time enters through the implicit function theorem on |dx + t dv| = R;
 * the periodic wrap has derivative 1. Returns -1 on a pair without a root. */
int or_collide_adjoint(int64_t n, const double* x, const double* v, const double* r, const double* m,
                       const int64_t* partner, double e, double dt, const double* gx_out, const double* gv_out,
                       double* gx_in, double* gv_in);

/* Vector-Jacobian product of or_project (affine mesh): given G = dL/dfield,
 * gq[c][p] = sum_g G[g][c] K_pg / Z_p and gx[a][p] = dL/dx_p (the kernel's
 * Gaussian derivative K (X - x)/sigma^2 inside the cutoff, Z_p differentiated
 * too; the cutoff itself is held fixed). */
int or_project_adjoint(int64_t n, const double* x, const double* q, int ne, int degree, double sigma,
                       double cutoff_sigmas, int cutoff_kind, const double* G, double* gq, double* gx);

/* Physical position of a logical point xi in [0,1)^3 under the periodic mesh
 * mapping x = xi + amp*(sin 2pi xi_y sin 2pi xi_z, sin 2pi xi_z sin 2pi xi_x,
 * sin 2pi xi_x sin 2pi xi_y) (amp = 0 is the affine Cartesian mesh), and the
 * determinant of its Jacobian. */
void or_mesh_map(const double xi[3], double amp, double X[3], double* detJ);

/* Projection of particle sources onto the Gauss nodes (Sec. 2.3 / 4.2 with a
 * Gaussian shape function): F[g,c] = sum_p q[c,p] K(X_g - x_p) / Z_p with
 * Z_p = sum_g W_g K(X_g - x_p), W_g = w_i w_j w_k (h/2)^3 det J at the node,
 * K(d) = exp(-|d|^2 / (2 sigma^2)) inside the cutoff and 0 outside.
 * cutoff_kind 0: box |d_axis| <= cutoff_sigmas*sigma on every axis;
 * 1: sphere |d| <= cutoff_sigmas*sigma. d is the periodic minimum image.
 * Sums use Neumaier compensated summation. Z (length n) may be NULL.
 * Returns 0 on success, nonzero on bad input or allocation failure. */
int or_project(int64_t n, const double* x, const double* q, int ne, int degree, double sigma, double cutoff_sigmas,
               int cutoff_kind, double amp, double* field, double* Z);

/* Linear corner-node deposition (Sec. 2.3, the deposition operator P in its linear
 * inverse-distance-weighting form; Sec. 4.2, unique periodic corner-node ids) on
 * the affine mesh: a particle at reference position xi of its element adds
 * q_c w_n(xi) to each of the element's 8 corner nodes, w_n(xi) = prod_d
 * (1 + s_d xi_d)/2 (s_d = -1/+1 for the lower/upper corner); node n carries the
 * density S_n / V_n with V_n = sum over the elements around n of the quadrature
 * sum_g W_g w_n(xi_g) (its Jacobian-weighted volume); the field at the Gauss
 * nodes of an element is the trilinear interpolation of its corner densities,
 * so sum_g W_g F_gc = sum_p q_pc. Neumaier sums. Returns 0 on success. */
int or_project_idw(int64_t n, const double* x, const double* q, int ne, int degree, double* field);

/* Dirac deposition (Sec. 4.2): the whole source of a particle goes to the Gauss
 * node of its element nearest in reference coordinates (per axis; the lower index
 * on a tie), as the density q / W_g. Returns 0 on success. */
int or_project_dirac(int64_t n, const double* x, const double* q, int ne, int degree, double* field);

/* The DG solution at the particles (Sec. 3.2, field evaluation): for each particle
 * in element e at reference position xi, out[c][p] = sum_{ijk} U[e][c][k][j][i]
 * l_i(xi_1) l_j(xi_2) l_k(xi_3), l the Lagrange basis of the Legendre-Gauss nodes;
 * field [ne^3][nvar][(N+1)^3]. Neumaier sums. Returns 0 on success. */
int or_eval_field(int64_t n, const double* x, const double* field, int ne, int degree, int nvar, double* out);

/* Momentum and energy sources of the drag force (Sec. 2.2 particle momentum
 * equation, Sec. 2.3 source terms): F = 3 pi mu_f d f_D (u_f - v_p), d = 2r, with the
 * Schiller-Naumann factor f_D = 1 + 0.15 Re^0.687, Re = rho_f |u_f - v_p| d / mu_f
 * (the paper's Loth correlation is not printed); q = (-F, -F.v_p) [4][n].
 * fluid [4][n] = (rho_f, u_f) at the particles. */
void or_drag_sources(int64_t n, const double* v, const double* r, const double* fluid, double mu_f, double* q);

#ifdef __cplusplus
}
#endif
#endif
