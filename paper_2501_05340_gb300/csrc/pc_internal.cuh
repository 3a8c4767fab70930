// Internal declarations of the pc library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>
#include <stdio.h>

#include "df32.cuh"
#include "pc.h"

// Device counters of one pc_collide / pc_project (64-bit, atomically updated).
enum {
  CNT_PAIRS = 0,
  CNT_CANDS,
  CNT_WORK,
  CNT_ROUNDS,
  CNT_SOLVES,
  CNT_MAXCAND,
  CNT_STENCIL,
  CNT_STATUS,  // pc_status raised on the GPU (max of codes)
  CNT_VMAX2,   // max |v|^2 as the bits of a non-negative double
  CNT_RMAX,    // max r as the bits of a non-negative double
  CNT_ELEM,    // next element of the mixed deposit (zeroed before each launch)
  CNT_RESP,    // colliding particles listed by the FP32 response
  CNT_N
};

#define PC_EVPOOL 4096

struct pc_ctx {
  pc_config cfg;
  cudaStream_t stream;
  int device;
  // collision cells
  int nc;
  int64_t ncell;
  // projection geometry
  int n1;
  int rho;   // neighbour elements searched on each side
  int win;   // factor window per axis: (2 rho + 1) n1 nodes
  double h;
  // binning scratch (shared by collide and project; sized for the larger grid)
  int64_t nbins_max;
  int32_t *cnt, *start, *blocksums;
  int32_t *key, *slot, *perm;
  // collide scratch (sorted order)
  double *sx, *sv, *sr;
  int32_t* sid;
  float *sxf, *svf, *srf;
  int32_t cap;
  int32_t* cand_j;
  double* cand_t;
  int32_t *ncand, *best, *partner, *work;
  int32_t* scell;  // sorted linear cells (mixed path)
  double* tcoll;
  int32_t *pair_lo, *pair_hi;
  double* pair_t;
  unsigned long long* counters;    // device [CNT_N]
  unsigned long long* h_counters;  // pinned host copy
  // projection scratch
  float2* fac;  // [3][win][n_max] normalised 1-D kernel factors (df32), sorted order
  float2* sq;   // [4][n_max] sources times (2/h)^3 (df32), sorted order
  // for n1 <= 8 fac holds records instead: [n_max][rs], rs = 3 win + 4 rounded up to
  // even (the window factors of the 3 axes, then the sources), for the tensor-core deposit
  int rs;
  int32_t* reach;   // [n_max] per-axis reach bits of the records
  unsigned* fxmax;  // [8]: largest factor and largest |source c| (float bits)
  DfExpTable exp_tab;
  int pair_policy;  // PC_PAIRS_EARLIEST or PC_PAIRS_SFC_FIRST (pc_set_pair_policy)
  double* corner;  // 36 ne^3 doubles: pc_project_idw's df32 corner sums [ne^3][8][4] and node densities [ne^3][4]
  float2* trig;    // [(ne + 2 rho) n1]: sin and cos of 2 pi X at the Gauss coordinates X = (e + s_i) h of
                   // one axis, with rho elements of periodic images either side
  // Legendre-Gauss nodes and weights (passed to the kernels as arguments)
  double eta[16], w[16];
  // per-phase timers (pc_set_timing) and the launch counter
  int timing;
  cudaEvent_t* ev;  // [2 * PC_EVPOOL], created when timing is first switched on
  int nrec;
  unsigned char rec_phase[PC_EVPOOL];
  int64_t launches;
  char err[256];
};

// Start a timed phase: returns the record index, or -1 when timing is off or full.
static inline int pc_phase_begin(pc_ctx* c, int phase) {
  if (!c->timing || !c->ev || c->nrec >= PC_EVPOOL) return -1;
  const int i = c->nrec++;
  c->rec_phase[i] = (unsigned char)phase;
  cudaEventRecord(c->ev[2 * i], c->stream);
  return i;
}
static inline void pc_phase_end(pc_ctx* c, int i) {
  if (i >= 0) cudaEventRecord(c->ev[2 * i + 1], c->stream);
}

// ---- binning (bin.cu) --------------------------------------------------------
// Exclusive scan of in[0..n) into out[0..n], out[n] = total. blocksums holds
// ceil(n / PC_SCAN_TILE) entries.
#define PC_SCAN_TILE 2048
cudaError_t pc_exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* blocksums, cudaStream_t s,
                              int64_t* launches);
// Given key[i] (bin) and slot[i] (rank inside its bin in arbitrary order), write the
// permutation sorted by (bin, id): perm[k] = input index of the k-th particle.
cudaError_t pc_bin_finish(int64_t n, int64_t nbins, const int32_t* key, const int32_t* slot, const int32_t* id,
                          int32_t* cnt, int32_t* start, int32_t* blocksums, int32_t* perm, cudaStream_t s,
                          int64_t* launches);

// ---- tables (pc_abi.cu) -----------------------------------------------------
void pc_gauss_rule(int n1, double* x, double* w);
void pc_build_exp_table(DfExpTable* tab);

// ---- collide (collide.cu) ----------------------------------------------------
// w_in / w_out: angular velocities [3][n] (input / output order) for the response with
// friction and rotation; NULL for the frictionless response.
pc_status pc_collide_impl(pc_ctx* ctx, const pc_particles* in, pc_particles* out, double dt,
                          const double* w_in = nullptr, double* w_out = nullptr, double mu = 0.0);
// Matching rounds on the candidate lists left by a search kernel (both paths).
cudaError_t pc_match_launch(pc_ctx* ctx, int64_t n);

// ---- mixed-precision path (mixed.cu, tc_deposit.cu) --------------------------
pc_status pc_quantize_impl(pc_ctx* ctx, const pc_particles* in, pc_particles_f32* out);
pc_status pc_collide_f32_impl(pc_ctx* ctx, const pc_particles_f32* in, pc_particles_f32* out, double dt);
pc_status pc_project_f32_impl(pc_ctx* ctx, const pc_particles_f32* p, float* field, int tc_type);
pc_status pc_collide_replay_f32_impl(pc_ctx* ctx, const pc_particles_f32* in, pc_particles_f32* out,
                                     const int32_t* partner, double dt);
pc_status pc_collide_adjoint_f32_impl(pc_ctx* ctx, const pc_particles_f32* in, const int32_t* partner, double dt,
                                      const float* gx_out, const float* gv_out, float* gx_in, float* gv_in);
pc_status pc_project_adjoint_f32_impl(pc_ctx* ctx, const pc_particles_f32* p, const float* G, float* gq,
                                      float* gx);
pc_status pc_project_curved_f32_impl(pc_ctx* ctx, const pc_particles_f32* p, float* field);
// Tensor-core deposit over the prepared particle records (tc_deposit.cu).
struct TcDepositArgs {
  int64_t n;
  int ne, n1, rho, tc_type;
  float c2l;        // h^2 / (2 sigma^2) log2(e): exponent factor for exp2 in element units
  float rce;        // cutoff in element units
  float scale_out;  // (2/h)^3 / (operand scalings)
  float s[16];      // (eta_i + 1) / 2
  const int32_t* start;
  const float4* rec;  // [n][4]: (t0 t1 t2 iz0) (iz1 iz2 q0 q1) (q2 q3 mask0 mask1) (mask2 reach - -)
  float* field;
  unsigned long long* counters;
};
cudaError_t pc_tc_deposit_launch(const TcDepositArgs& A, cudaStream_t st, int* nblocks);

// FP64-accurate tensor-core deposit over the records of k_proj_factors (fx_deposit.cu).
cudaError_t pc_fx_deposit_launch(int n1, int ne, int rho, int win, int rs, const int32_t* start, const float2* rec,
                                 const int32_t* reach, const unsigned* fxmax, double* field,
                                 unsigned long long* counters, cudaStream_t st);

// ---- project (project.cu) ----------------------------------------------------
pc_status pc_project_impl(pc_ctx* ctx, const pc_particles* p, double* field);
// Particles binned by mesh element: ctx->start[e] .. ctx->start[e + 1] index
// ctx->perm, which lists the input indices of element e's particles in id order.
// Positions outside [0,1) raise PC_EINVAL in the device status.
cudaError_t pc_elem_bin(pc_ctx* ctx, int64_t n, const double* x, const int32_t* id);

// ---- fluid -> particle coupling (coupling.cu) ----------------------------------
pc_status pc_eval_field_impl(pc_ctx* ctx, const pc_particles* p, const double* field, int nvar, double* out);
pc_status pc_drag_sources_impl(pc_ctx* ctx, const pc_particles* p, const double* fluid, double mu_f, double* q);

// ---- corner-node and nearest-DOF depositions (nodal.cu) -----------------------
pc_status pc_project_idw_impl(pc_ctx* ctx, const pc_particles* p, double* field);
pc_status pc_project_dirac_impl(pc_ctx* ctx, const pc_particles* p, double* field);

#define PC_CUDA_TRY(expr)                          \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return _e;              \
  } while (0)

static inline int pc_blocks(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

#ifdef __CUDACC__
// Maxima of two non-negative doubles over the block into two counters (their bit
// patterns order like the values): one atomic per block and counter, skipped when the
// counter already holds as much (a stale read only costs the atomic). Every thread of
// the block calls it; every counter update of one address from all warps of a large
// grid would serialise in the L2.
__device__ __forceinline__ void pc_block_max2(unsigned long long* c0, double v0, unsigned long long* c1, double v1) {
  __shared__ double red[2][32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 = fmax(v0, __shfl_xor_sync(0xffffffffu, v0, o));
    v1 = fmax(v1, __shfl_xor_sync(0xffffffffu, v1, o));
  }
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = v0;
    red[1][w] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < nw; ++i) {
      v0 = fmax(v0, red[0][i]);
      v1 = fmax(v1, red[1][i]);
    }
    const unsigned long long b0 = (unsigned long long)__double_as_longlong(v0);
    const unsigned long long b1 = (unsigned long long)__double_as_longlong(v1);
    if (b0 > *(volatile unsigned long long*)c0) atomicMax(c0, b0);
    if (b1 > *(volatile unsigned long long*)c1) atomicMax(c1, b1);
  }
}
#endif
