// FP64-accurate deposit of the projection on the tensor cores (tcgen05, sm_103a),
// by exact fixed-point digits (arXiv 2501.05340 Sec. 2.3 source terms, Sec. 4.2
// deposition, with the Gaussian shape function of pc_project).
//
// For one element with n1 = N+1 <= 8 Gauss nodes per axis the separable deposit is
//   D[jk][c i] = sum_p YZ[p][jk] A[p][c i],  YZ = ky_j kz_k,  A = q_c kx_i,
// a dense contraction over the particles p whose support reaches the element. The
// factors are double-float (about 48 bits). Each product value v (YZ or A) is
// scaled by a power of two common to all particles (|v| < 1/2) and written as
//   v = sum_{d=0..5} s_d 2^(-8 (d+1)) + r,   s_d integers, |r| <= 2^-49,
// with |s_d| <= 128 except |s_3| <= 512, so every digit is exact in FP16. The
// tensor core multiplies digit matrices and sums the products in FP32. The cells
// whose weight is within 2^-16 of the leading one (r + b <= 2 below) take at most
// two products of digits 0..2 (each at most 2^14 in magnitude) per particle, so
// their sums stay below 2^24 and are exact, whatever the order, for up to 1024
// particles (512 when two products meet in one cell); the other cells weigh 2^-24
// or less of the leading one, where FP32 rounding stays below 2^-46 of the result.
// The deposit is
//   D = 2^(EY + EA) sum_{a,b} 2^(-8 (a + b + 2)) sum_p Y_a[p] A_b[p].
//
// Tensor layout: the A operand (M = 128 rows) of MMA group g holds the YZ digits
// a = R g .. R g + R - 1 (R = floor(128 / n1^2) digit blocks of n1^2 rows); the B
// operand holds the A digits b = 0..5 (blocks of CP >= 4 n1 rows) and MMA group g
// writes the accumulator columns from R g CP on. Accumulator cell (r, b) (row block
// r, column block b) then sums Y_(Rg+r) A_(b-Rg) over all groups g: every product
// in a cell has the weight 2^(-8 (r + b + 2)). The epilogue adds the cells with
// their weights in double-float arithmetic and writes FP64.
//
// Warp roles of the persistent CTA (one per SM, all 512 tensor-memory columns as
// two 256-column accumulators so that one element drains while the next
// accumulates): 8 gather warps take the element's candidate particles in batches
// of 32 in a fixed order, keep those whose support reaches the element (per-axis
// reach bits) and stage their factors; 9 builder warps, in three teams of three
// that take every third batch, turn a staged batch into the digit operands; one MMA warp
// issues the MMAs of each batch in batch order
// (so the result does not depend on scheduling) and hands finished elements to 4
// epilogue warps (one per tensor-memory lane quarter). An element with more kept
// particles than one segment holds is deposited in segments added in FP64. Every wait
// is bounded in wall-clock time: on expiry the kernel records PC_ETIMEOUT, stops
// issuing, waits (bounded) for its MMAs and frees its tensor memory.
#include <cuda_fp16.h>
#include <stdint.h>

#include "pc_internal.cuh"

namespace {

constexpr int kS = 6;                                 // digits per value
constexpr float kBase = 256.0f;                       // digit radix (8 bits)
constexpr float kInvBase = 1.0f / 256.0f;
constexpr int kGather = 8;                            // gather warps
constexpr int kBuild = 9;                             // builder warps
constexpr int kTeams = 3;                             // builder teams, each on every kTeams-th batch
constexpr int kTeamWarps = kBuild / kTeams;
constexpr int kEpi = 4;                               // epilogue warps
constexpr int kWarps = 1 + kEpi + kGather + kBuild;   // + the MMA warp
constexpr int kThreads = 32 * kWarps;
constexpr int kQ = 16;                                // finished-job queue
constexpr int kMaxRanges = 125;                       // (2 rho + 1)^3 neighbour elements, rho <= 2
constexpr int kFRow = 34;                             // staged row pitch in float2 (272 B: rows 16 B apart in the banks)
constexpr unsigned long long kWaitNs = 2000000000;    // a wait without progress for 2 s fails
constexpr size_t kSmemMax = 232448;                   // 227 KB per CTA

__host__ __device__ constexpr int rup(int a, int m) { return (a + m - 1) / m * m; }

template <int N1>
struct FxShape {
  static constexpr int JK = N1 * N1;                       // YZ rows per digit
  static constexpr int CI = 4 * N1;                        // A columns per digit
  static constexpr int CP = rup(CI, 8);                    // A digit block (whole core matrices)
  static constexpr int R = (128 / JK) < kS ? 128 / JK : kS; // YZ digits per MMA group
  static constexpr int G = (kS + R - 1) / R;               // MMA groups
  static constexpr int BR = rup(kS * CP, 16);              // B operand rows
  static constexpr int NFLD = 3 * N1 + 4;                  // staged df32 fields per particle
  static constexpr int ATILE = 128 * 64;                   // bytes: 128 rows x 32 K x FP16
  static constexpr int STAGE = G * ATILE + BR * 64;
  static constexpr int FSLOT = NFLD * kFRow * 8;
  static constexpr int COMB = R * JK * CI * 8;
  static constexpr int NA = 4 * rup(JK, 8);                // YZ build items: (jk, particle octet)
  static constexpr int NB = 4 * rup(CI, 8);                // A build items: (ci, particle octet)
  static constexpr int FIXED = COMB + kGather * (3 * kMaxRanges + 1) * 4 + 4096;
  static constexpr int NF = 8;                             // staged-factor slots
  static constexpr int NS0 = (int)((kSmemMax - 1024 - FIXED - NF * FSLOT) / STAGE);
  static constexpr int NS = NS0 > 4 ? 4 : NS0;             // operand stages
  // kept particles per accumulation segment: the exact cells hold one digit product
  // per particle when R >= 3 and two when R = 2
  static constexpr int SEG = R >= 3 ? 1024 : 512;
  __host__ __device__ static constexpr int ncol(int g) { return rup(CP * (kS - R * g), 16); }
  __host__ __device__ static constexpr int col0(int g) { return R * g * CP; }
};

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets, fixed version bits 46-48 = 0b001, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major operand tile of 32 K values per row, no swizzle: 8-row x 16-byte core
// matrices, (row/8) * 512 + (k/8) * 128 + (row%8) * 16 + (k%8) * 2.
__device__ __forceinline__ int kmaj32(int row, int k) {
  return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int vload(const int* p) { return *(const volatile int*)p; }

__device__ __forceinline__ bool mbar_try(unsigned long long* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

constexpr uint32_t kSuspendNs = 100000;
__device__ __forceinline__ bool mbar_try_sleep(unsigned long long* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Shared state besides the operand stages, factor slots and the epilogue's
// combination buffer (carved from dynamic shared memory after this struct).
struct FxCtl {
  unsigned long long f_full[8], f_empty[8];    // factor slots: gather -> builders
  unsigned long long op_full[4], op_empty[4];  // operand stages: builders -> MMA (tcgen05.commit)
  unsigned long long acc_full[2], acc_empty[2];
  unsigned long long qfull[kQ], qempty[kQ];
  unsigned long long fin;
  int fmeta[8][4];   // element (-1 ends the stream), kept count, first batch, last batch
  __align__(16) int opmeta[4][4];
  int qe[kQ], qslot[kQ], qseg[kQ];
  int failed;
  int progress;
  int ey, ec[4];     // digit scales: |YZ| / 2^ey and |A_c| / 2^ec[c] are below 1/2
  uint32_t tmem_base;
};

// Waits for the phase of the given parity. Returns false once the block has failed,
// or after kWaitNs in which no gather warp reported progress. With backoff the warp
// sleeps between polls (for waits that usually last microseconds), so that idle
// warps leave the issue slots and the shared-memory pipe to the working ones.
__device__ bool fx_wait(FxCtl& C, unsigned long long* bar, uint32_t parity, bool backoff = false) {
  if (mbar_try(bar, parity)) return true;
  unsigned long long t0 = gtime();
  int last = -1;
  unsigned ns = 64;
  for (int it = 1;; ++it) {
    if (backoff) {
      __nanosleep(ns);
      if (ns < 1024) ns *= 2;
      if (mbar_try(bar, parity)) return true;
    } else if (mbar_try_sleep(bar, parity)) {
      return true;
    }
    if ((it & 15) == 0) {
      if (vload(&C.failed)) return false;
      const unsigned long long now = gtime();
      if (now - t0 > kWaitNs) {
        const int p = vload(&C.progress);
        if (p == last) return false;
        last = p;
        t0 = now;
      }
    }
  }
}

__device__ __forceinline__ void fail_now(FxCtl& C, unsigned long long* counters) {
  *(volatile int*)&C.failed = 1;
  atomicMax(&counters[CNT_STATUS], (unsigned long long)PC_ETIMEOUT);
}

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

struct FxArgs {
  int ne, rho, win, rs;
  int64_t nel;
  const int32_t* start;
  const float2* rec;
  const int32_t* reach;
  const unsigned* fxmax;
  double* field;
  unsigned long long* counters;
};

template <int N1>
struct FxSmem {
  using B = FxShape<N1>;
  uint8_t* stage;   // [NS][G ATILE + BR 64]
  float2* fslot;    // [NF][NFLD][kFRow]
  float2* comb;     // [R JK][CI] df32
  int* pre;         // [kGather][kMaxRanges + 1]
  int* rbeg;        // [kGather][kMaxRanges]
  int* rmeta;       // [kGather][kMaxRanges]
  FxCtl* ctl;
};

// Gather warp w: batches q = w, w + kGather, ... of the CTA's stream (elements
// blockIdx.x + m gridDim.x, each in batches of 32 candidates; an element without
// candidates still has one, empty, batch).
template <int N1>
__device__ void fx_gather(const FxSmem<N1>& M, const FxArgs& A, int w, int lane) {
  using B = FxShape<N1>;
  FxCtl& C = *M.ctl;
  const int ne = A.ne, rho = A.rho, span = 2 * rho + 1, nrange = span * span * span;
  int* pre = M.pre + w * (kMaxRanges + 1);
  int* rbeg = M.rbeg + w * kMaxRanges;
  int* rmeta = M.rmeta + w * kMaxRanges;
  // digit scales of the four sources and of YZ
  const float sy = ldexpf(1.0f, -C.ey);
  float sc[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) sc[c] = ldexpf(1.0f, -C.ec[c]);
  int64_t q = 0;  // first batch of the current element
  bool ok = true;
  for (int64_t e = blockIdx.x; ok && e < A.nel; e += gridDim.x) {
    const int ex = (int)(e % ne), ey = (int)((e / ne) % ne), ez = (int)(e / ((int64_t)ne * ne));
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
        rmeta[r] = (rho - dx) | ((rho - dy) << 8) | ((rho - dz) << 16);
      }
      int x = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (r < nrange) pre[r + 1] = total + x;
      total += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) pre[0] = 0;
    __syncwarp();
    const int nb = total > 0 ? (total + 31) / 32 : 1;
    int top = 1;
    while (2 * top < nrange) top *= 2;
    for (int b = (int)((w - q % kGather + kGather) % kGather); b < nb; b += kGather) {
      const int64_t qq = q + b;
      const int fs = (int)(qq % B::NF);
      if (qq >= B::NF && !fx_wait(C, &C.f_empty[fs], (uint32_t)(((qq / B::NF) - 1) & 1), true)) {
        if (lane == 0) fail_now(C, A.counters);
        ok = false;
        break;
      }
      const int idx = b * 32 + lane;
      bool kept = false;
      int64_t j = 0;
      int wm = 0;
      if (idx < total) {
        int r = 0;
        for (int stp = top; stp > 0; stp >>= 1)
          if (r + stp < nrange && pre[r + stp] <= idx) r += stp;
        j = rbeg[r] + (idx - pre[r]);
        wm = rmeta[r];
        const int bits = A.reach[j];
        kept = ((bits >> (wm & 255)) & (bits >> (8 + ((wm >> 8) & 255))) & (bits >> (16 + ((wm >> 16) & 255))) & 1) !=
               0;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, kept);
      const int nk = __popc(bal);
      float2* fst = M.fslot + (size_t)fs * B::NFLD * kFRow;
      if (kept) {
        const int pos = __popc(bal & ((1u << lane) - 1u));
        const float2* rp = A.rec + j * A.rs;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float2* src = rp + a * A.win + ((wm >> (8 * a)) & 255) * N1;
          const float s = a == 1 ? sy : 1.0f;
#pragma unroll
          for (int i = 0; i < N1; ++i) {
            const float2 v = src[i];
            fst[(a * N1 + i) * kFRow + pos] = make_float2(v.x * s, v.y * s);
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float2 v = rp[3 * A.win + c];
          fst[(3 * N1 + c) * kFRow + pos] = make_float2(v.x * sc[c], v.y * sc[c]);
        }
      }
      if (lane >= nk) {
#pragma unroll
        for (int f = 0; f < B::NFLD; ++f) fst[f * kFRow + lane] = make_float2(0.0f, 0.0f);
      }
      if (lane == 0) {
        C.fmeta[fs][0] = (int)e;
        C.fmeta[fs][1] = nk;
        C.fmeta[fs][2] = b == 0;
        C.fmeta[fs][3] = b == nb - 1;
        atomicAdd(&C.progress, 1);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&C.f_full[fs]);
    }
    q += nb;
  }
  // end of the stream: one end marker per builder team (batches q .. q + kTeams - 1),
  // each written by the warp that owns its batch
  for (int x = 0; ok && x < kTeams; ++x) {
    const int64_t qq = q + x;
    if (qq % kGather != w) continue;
    const int fs = (int)(qq % B::NF);
    const bool free_slot = qq < B::NF || fx_wait(C, &C.f_empty[fs], (uint32_t)(((qq / B::NF) - 1) & 1), true);
    if (lane == 0) {
      if (!free_slot) fail_now(C, A.counters);
      C.fmeta[fs][0] = -1;
      mbar_arrive(&C.f_full[fs]);
    }
  }
}

// Digits of a value v = y + w (|v| < 1/2, y the high and w the low part of a
// double-float product, |w| <= 3 2^-24 |y|): s_d = rint of the remainder scaled by
// 256^(d+1). The first three come from y alone, exactly (y holds 24 bits); then w
// joins the remainder, whose rounding there is below 2^-47 of v's scale. |s_3| <=
// 512, the others <= 128; the remainder after six digits is below 2^-49.

// Builder warp bi: digit operands of the batches of its team (bi % kTeams), in batch
// order; the teams build consecutive batches at the same time.
template <int N1>
__device__ void fx_build(const FxSmem<N1>& M, const FxArgs& A, int bi, int lane) {
  using B = FxShape<N1>;
  FxCtl& C = *M.ctl;
  const int team = bi % kTeams, tw = bi / kTeams;
  for (int64_t q = team;; q += kTeams) {
    const int fs = (int)(q % B::NF);
    const int os = (int)(q % B::NS);
    if (!fx_wait(C, &C.f_full[fs], (uint32_t)((q / B::NF) & 1))) {
      if (lane == 0) fail_now(C, A.counters);
      return;
    }
    const int e = C.fmeta[fs][0], nk = C.fmeta[fs][1];
    if (q >= B::NS && !fx_wait(C, &C.op_empty[os], (uint32_t)(((q / B::NS) - 1) & 1))) {
      if (lane == 0) fail_now(C, A.counters);
      return;
    }
    if (e >= 0 && nk > 0) {
      const float2* fst = M.fslot + (size_t)fs * B::NFLD * kFRow;
      uint8_t* stg = M.stage + (size_t)os * B::STAGE;
      const int nok = nk > 16 ? 4 : 2;  // particle octets the MMAs read
      for (int it = tw * 32 + lane; it < B::NA + B::NB; it += kTeamWarps * 32) {
        const bool isA = it < B::NA;
        const int t = isA ? it : it - B::NA;
        const int row = 8 * (t >> 5) + (t & 7), o = (t >> 3) & 3;
        if (o >= nok || row >= (isA ? B::JK : B::CI)) continue;
        // the 8 values of this row for particles 8 o .. 8 o + 7, as 4 pairs of
        // neighbouring particles on the packed FP32x2 instructions
        float2 vy[4], vw[4];
        const float2* f0;
        const float2* f1;
        if (isA) {
          f0 = fst + (N1 + row % N1) * kFRow + 8 * o;      // ky_j
          f1 = fst + (2 * N1 + row / N1) * kFRow + 8 * o;  // kz_k
        } else {
          f0 = fst + (3 * N1 + row / N1) * kFRow + 8 * o;  // q_c
          f1 = fst + (row % N1) * kFRow + 8 * o;           // kx_i
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 a4 = *reinterpret_cast<const float4*>(f0 + 2 * u);
          const float4 b4 = *reinterpret_cast<const float4*>(f1 + 2 * u);
          // double-float products (a.h + a.l)(b.h + b.l) as an unevaluated high + low pair
          const float2 ah = make_float2(a4.x, a4.z), al = make_float2(a4.y, a4.w);
          const float2 bh = make_float2(b4.x, b4.z), bl = make_float2(b4.y, b4.w);
          const float2 p = __fmul2_rn(ah, bh);
          float2 l = __ffma2_rn(ah, bh, make_float2(-p.x, -p.y));
          l = __ffma2_rn(ah, bl, l);
          vy[u] = p;
          vw[u] = __ffma2_rn(al, bh, l);
        }
        // digits, one per particle and step (see the note above); the first three from
        // the high parts alone, then the low parts join
        const float2 Mg = make_float2(12582912.0f, 12582912.0f);  // 1.5 * 2^23: adding it rounds to an integer
        const float2 nMg = make_float2(-12582912.0f, -12582912.0f);
        const float2 base2 = make_float2(kBase, kBase);
        const float2 b32 = make_float2(4294967296.0f, 4294967296.0f);
#pragma unroll
        for (int u = 0; u < 4; ++u) vy[u] = __fmul2_rn(vy[u], base2);
#pragma unroll
        for (int k = 0; k < kS; ++k) {
          uint32_t h[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (k == 3) vy[u] = __ffma2_rn(vw[u], b32, vy[u]);
            const float2 dg = __fadd2_rn(__fadd2_rn(vy[u], Mg), nMg);
            vy[u] = __fmul2_rn(__fadd2_rn(vy[u], make_float2(-dg.x, -dg.y)), base2);
            const __half2 v = __floats2half2_rn(dg.x, dg.y);
            h[u] = *reinterpret_cast<const uint32_t*>(&v);
          }
          int off;
          if (isA)
            off = (k / B::R) * B::ATILE + kmaj32((k % B::R) * B::JK + row, 8 * o);
          else
            off = B::G * B::ATILE + kmaj32(k * B::CP + row, 8 * o);
          *reinterpret_cast<uint4*>(stg + off) = make_uint4(h[0], h[1], h[2], h[3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();
    if (lane == 0) {
      if (tw == 0) {
#pragma unroll
        for (int x = 0; x < 4; ++x) C.opmeta[os][x] = C.fmeta[fs][x];
      }
      mbar_arrive(&C.f_empty[fs]);
      mbar_arrive(&C.op_full[os]);
    }
    if (e < 0) return;
  }
}

// Job queue MMA warp -> epilogue: entry t is reused once the epilogue warps have
// read entry t - kQ.
__device__ __forceinline__ bool queue_push(FxCtl& C, int t, int e, int slot, int seg) {
  if (t >= kQ && !fx_wait(C, &C.qempty[t % kQ], (uint32_t)(((t / kQ) - 1) & 1))) return false;
  C.qe[t % kQ] = e;
  C.qslot[t % kQ] = slot;
  C.qseg[t % kQ] = seg;
  mbar_arrive(&C.qfull[t % kQ]);
  return true;
}

// MMA warp (lane 0 issues): the batches in order; an element's MMAs accumulate in
// one of the two tensor-memory accumulators, which alternate between jobs.
template <int N1>
__device__ void fx_mma(const FxSmem<N1>& M, const FxArgs& A, uint32_t tmem, int lane) {
  using B = FxShape<N1>;
  FxCtl& C = *M.ctl;
  if (lane == 0) {
    int slot = 0, uses[2] = {0, 0}, t = 0, seg = 0, kept = 0;
    bool started = false, failed = false;
    // descriptors of stage 0; stage s differs only in the start address field
    const uint32_t sa0 = smem_u32(M.stage);
    uint64_t da0[B::G][2], db0[2];
    uint32_t idesc[B::G];
#pragma unroll
    for (int g = 0; g < B::G; ++g) {
      idesc[g] = (1u << 4) | ((uint32_t)(B::ncol(g) >> 3) << 17) | (8u << 24);
#pragma unroll
      for (int h = 0; h < 2; ++h) da0[g][h] = make_desc(sa0 + g * B::ATILE + 256 * h, 128, 512);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) db0[h] = make_desc(sa0 + B::G * B::ATILE + 256 * h, 128, 512);
    for (int64_t q = 0;; ++q) {
      const int os = (int)(q % B::NS);
      const uint32_t par = (uint32_t)((q / B::NS) & 1);
      if (!mbar_try(&C.op_full[os], par) && !fx_wait(C, &C.op_full[os], par)) {
        if (!vload(&C.failed)) fail_now(C, A.counters);
        failed = true;
        break;
      }
      const int4 mt = *reinterpret_cast<const int4*>(C.opmeta[os]);
      const int e = mt.x, nk = mt.y, first = mt.z, last = mt.w;
      if (e < 0) break;
      if (first) {
        seg = 0;
        kept = 0;
        started = false;
      }
      if (nk > 0) {
        if (started && kept + nk > B::SEG) {  // close the segment: its exact cells stay exact
          mma_commit(&C.acc_full[slot]);
          if (!queue_push(C, t++, e, slot, seg++)) {
            failed = true;
            break;
          }
          slot ^= 1;
          started = false;
          kept = 0;
        }
        if (!started && uses[slot] > 0 && !fx_wait(C, &C.acc_empty[slot], (uint32_t)((uses[slot] - 1) & 1))) {
          fail_now(C, A.counters);
          failed = true;
          break;
        }
        if (!started) ++uses[slot];
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t so = (uint64_t)((os * B::STAGE) >> 4);
        const uint32_t d0 = tmem + 256u * (uint32_t)slot;
#pragma unroll
        for (int g = 0; g < B::G; ++g)
          mma_f16(d0 + (uint32_t)B::col0(g), da0[g][0] + so, db0[0] + so, idesc[g], (started || g > 0) ? 1u : 0u);
        if (nk > 16) {
#pragma unroll
          for (int g = 0; g < B::G; ++g) mma_f16(d0 + (uint32_t)B::col0(g), da0[g][1] + so, db0[1] + so, idesc[g], 1u);
        }
        started = true;
        kept += nk;
      }
      mma_commit(&C.op_empty[os]);
      if (last) {
        bool pushed;
        if (started) {
          mma_commit(&C.acc_full[slot]);
          pushed = queue_push(C, t++, e, slot, seg);
          slot ^= 1;
        } else {
          pushed = queue_push(C, t++, e, -1, 0);  // no particle reaches the element: zeros
        }
        if (!pushed) {
          failed = true;
          break;
        }
      }
    }
    if (failed && !vload(&C.failed)) fail_now(C, A.counters);
    // every MMA this thread issued has completed once this commit arrives
    mma_commit(&C.fin);
    const unsigned long long t0 = gtime();
    while (!mbar_try_sleep(&C.fin, 0) && gtime() - t0 < kWaitNs) {
    }
    if (!failed) queue_push(C, t, -1, -1, 0);
  }
  __syncwarp();
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t u[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
      : "r"(taddr));
}

// df32 a + b / 256 for an FP32 a and a df32 b.
__device__ __forceinline__ f2 horner_step(float a, f2 b) {
  const f2 s = two_sum(a, b.h * kInvBase);
  return fast_two_sum(s.h, s.l + b.l * kInvBase);
}

// Epilogue warp eq (tensor-memory lanes 32 (warp % 4) ..): drains the queue in order.
template <int N1>
__device__ void fx_epilogue(const FxSmem<N1>& M, const FxArgs& A, uint32_t tmem, int warp, int eq, int lane) {
  using B = FxShape<N1>;
  constexpr int NODES = N1 * N1 * N1;
  FxCtl& C = *M.ctl;
  const int quarter = warp & 3;
  const int row = 32 * quarter + lane;
  const int r = row / B::JK, jk = row - r * B::JK;
  const bool rvalid = r < B::R;
  int seen[2] = {0, 0};
  for (int t = 0;; ++t) {
    if (!fx_wait(C, &C.qfull[t % kQ], (uint32_t)((t / kQ) & 1), true)) {
      if (lane == 0 && eq == 0 && !vload(&C.failed)) fail_now(C, A.counters);
      return;
    }
    const int e = C.qe[t % kQ], slot = C.qslot[t % kQ], seg = C.qseg[t % kQ];
    __syncwarp();
    if (lane == 0) mbar_arrive(&C.qempty[t % kQ]);
    if (e < 0) return;
    if (slot >= 0) {
      if (!fx_wait(C, &C.acc_full[slot], (uint32_t)(seen[slot] & 1), true)) {
        if (lane == 0 && !vload(&C.failed)) fail_now(C, A.counters);
        return;
      }
      ++seen[slot];
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ta = tmem + 256u * (uint32_t)slot + ((uint32_t)(32 * quarter) << 16);
#pragma unroll 1
      for (int cb = 0; cb < B::CP / 8; ++cb) {
        uint32_t u[kS][8];
#pragma unroll
        for (int b = 0; b < kS; ++b) tmem_ld8(ta + (uint32_t)(b * B::CP + 8 * cb), u[b]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const int ci = 8 * cb + x;
          f2 P = {__uint_as_float(u[kS - 1][x]), 0.0f};
#pragma unroll
          for (int b = kS - 2; b >= 0; --b) P = horner_step(__uint_as_float(u[b][x]), P);
          if (rvalid && ci < B::CI) M.comb[(size_t)row * B::CI + ci] = make_float2(P.h, P.l);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&C.acc_empty[slot]);
      asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpi) : "memory");
    }
    // outputs: field[e][c][jk][i] = 2^(ey + ec - 16) sum_r 2^(-8 r) P_r[jk][c i]
    double* out = A.field + (int64_t)e * 4 * NODES;
    double sc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) sc[c] = ldexp(1.0, C.ey + C.ec[c] - 16);
    for (int o = eq * 32 + lane; o < 4 * NODES; o += 32 * kEpi) {
      const int c = o / NODES, rem = o - c * NODES, ojk = rem / N1, i = rem - ojk * N1;
      double val = 0.0;
      if (slot >= 0) {
        const int ci = c * N1 + i;
        f2 Q = {0.0f, 0.0f};
#pragma unroll
        for (int rr = B::R - 1; rr >= 0; --rr) {
          const float2 v = M.comb[(size_t)(rr * B::JK + ojk) * B::CI + ci];
          Q = df_add({v.x, v.y}, {Q.h * kInvBase, Q.l * kInvBase});
        }
        val = ((double)Q.h + (double)Q.l) * sc[c];
      }
      if (seg == 0)
        out[o] = val;
      else
        out[o] += val;
    }
    if (slot >= 0) asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpi) : "memory");
  }
}

template <int N1>
__global__ void __launch_bounds__(kThreads, 1) k_fx_deposit(FxArgs A) {
  using B = FxShape<N1>;
  static_assert(B::NS >= 2, "operand stages do not fit in shared memory");
  static_assert(B::NF <= 8 && B::NS <= 4, "more slots than the control block's barriers");
  static_assert(kBuild % kTeams == 0, "builder teams of unequal size");
  static_assert(B::R * B::JK <= 128, "YZ digit rows exceed the MMA's M");
  static_assert(B::col0(B::G - 1) + B::ncol(B::G - 1) <= 256 && B::ncol(0) <= 256, "accumulator wider than 256");
  extern __shared__ uint8_t smraw[];
  uint8_t* base = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  FxSmem<N1> M;
  M.stage = base;
  M.fslot = reinterpret_cast<float2*>(base + (size_t)B::NS * B::STAGE);
  M.comb = M.fslot + (size_t)B::NF * B::NFLD * kFRow;
  M.pre = reinterpret_cast<int*>(M.comb + (size_t)B::R * B::JK * B::CI);
  M.rbeg = M.pre + kGather * (kMaxRanges + 1);
  M.rmeta = M.rbeg + kGather * kMaxRanges;
  M.ctl = reinterpret_cast<FxCtl*>(M.rmeta + kGather * kMaxRanges);
  FxCtl& C = *M.ctl;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // zero the operand stages once: padding rows stay zero for good
  for (int i = tid; i < B::NS * B::STAGE / 16; i += kThreads)
    reinterpret_cast<uint4*>(M.stage)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < B::NF; ++s) {
      mbar_init(&C.f_full[s], 1);
      mbar_init(&C.f_empty[s], kTeamWarps);
    }
    for (int s = 0; s < B::NS; ++s) {
      mbar_init(&C.op_full[s], kTeamWarps);
      mbar_init(&C.op_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&C.acc_full[s], 1);
      mbar_init(&C.acc_empty[s], kEpi);
    }
    for (int s = 0; s < kQ; ++s) {
      mbar_init(&C.qfull[s], 1);
      mbar_init(&C.qempty[s], kEpi);
    }
    mbar_init(&C.fin, 1);
    C.failed = 0;
    C.progress = 0;
    // digit scales from the largest factor and sources: |v| / 2^E < 1/2 (frexp:
    // x < 2^ex); the margin covers the low parts of the double-float values
    const double fm = (double)__uint_as_float(A.fxmax[0]) * (1.0 + 1e-6);
    int ex = 0;
    frexp(fm * fm, &ex);
    C.ey = fm > 0.0 ? ex + 1 : 0;
    for (int c = 0; c < 4; ++c) {
      const double am = fm * (double)__uint_as_float(A.fxmax[1 + c]) * (1.0 + 1e-6);
      frexp(am, &ex);
      C.ec[c] = am > 0.0 ? ex + 1 : 0;
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&C.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = C.tmem_base;
  if (warp == 0)
    fx_mma<N1>(M, A, tmem, lane);
  else if (warp <= kEpi)
    fx_epilogue<N1>(M, A, tmem, warp, warp - 1, lane);
  else if (warp <= kEpi + kGather)
    fx_gather<N1>(M, A, warp - 1 - kEpi, lane);
  else
    fx_build<N1>(M, A, warp - 1 - kEpi - kGather, lane);
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

template <int N1>
size_t fx_smem() {
  using B = FxShape<N1>;
  return (size_t)B::NS * B::STAGE + (size_t)B::NF * B::FSLOT + (size_t)B::COMB +
         (size_t)kGather * (3 * kMaxRanges + 1) * 4 + sizeof(FxCtl) + 1024;
}

template <int N1>
cudaError_t fx_launch(const FxArgs& A, int sms, cudaStream_t st) {
  const size_t smem = fx_smem<N1>();
  if (smem > kSmemMax) return cudaErrorInvalidConfiguration;
  PC_CUDA_TRY(cudaFuncSetAttribute(k_fx_deposit<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int64_t grid = A.nel < sms ? A.nel : sms;
  if (grid < 1) grid = 1;
  k_fx_deposit<N1><<<(unsigned)grid, kThreads, smem, st>>>(A);
  return cudaGetLastError();
}

}  // namespace

// FP64-accurate tensor-core deposit for n1 = N + 1 <= 8 over the records written by
// k_proj_factors (record layout): field[e][c][k][j][i], overwritten.
cudaError_t pc_fx_deposit_launch(int n1, int ne, int rho, int win, int rs, const int32_t* start, const float2* rec,
                                 const int32_t* reach, const unsigned* fxmax, double* field,
                                 unsigned long long* counters, cudaStream_t st) {
  FxArgs A;
  A.ne = ne;
  A.rho = rho;
  A.win = win;
  A.rs = rs;
  A.nel = (int64_t)ne * ne * ne;
  A.start = start;
  A.rec = rec;
  A.reach = reach;
  A.fxmax = fxmax;
  A.field = field;
  A.counters = counters;
  int dev = 0, sms = 0;
  PC_CUDA_TRY(cudaGetDevice(&dev));
  PC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  switch (n1) {
    case 1: return fx_launch<1>(A, sms, st);
    case 2: return fx_launch<2>(A, sms, st);
    case 3: return fx_launch<3>(A, sms, st);
    case 4: return fx_launch<4>(A, sms, st);
    case 5: return fx_launch<5>(A, sms, st);
    case 6: return fx_launch<6>(A, sms, st);
    case 7: return fx_launch<7>(A, sms, st);
    case 8: return fx_launch<8>(A, sms, st);
    default: return cudaErrorInvalidValue;
  }
}
