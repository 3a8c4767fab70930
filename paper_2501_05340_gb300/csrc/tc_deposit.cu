// Tensor-core deposit of the mixed-precision projection (tcgen05, sm_103a).
//
// For one element with n1 = N+1 <= 8 Gauss nodes per axis the separable deposit is
//   D[jk][c i] = sum_p YZ[p][jk] A[p][c i],  YZ = ky_j kz_k,  A = q_c kx_i,
// a dense contraction over the particles p whose support reaches the element.
// Each factor is split into a high and a low part of the operand type (FP16 or
// BF16) and one MMA of M = 128, N = 64, K = 16 computes all four products at once:
//   A operand rows  0..63 : YZ_hi (scaled by 2^8), rows 64..127: YZ_lo
//   B operand rows  0..31 : A_hi  (scaled by 2^4), rows 32..63 : A_lo
// so D = [[hi hi, hi lo], [lo hi, lo lo]] accumulates in FP32 in tensor memory and
// the element's deposit is the sum of the four quadrants (the lo*lo one is below
// the accuracy of the others and harmless).
//
// Operands live in shared memory in the K-major layout without swizzle: core
// matrices of 8 rows x 16 bytes, (row/8) * 256 + (k/8) * 128 + (row%8) * 16 + (k%8) * 2.
// One elected thread issues tcgen05.mma and tcgen05.commit; the commit arrives on
// the stage's mbarrier when the tensor core has read the stage. Every wait on an
// mbarrier is bounded: on expiry the kernel records PC_ETIMEOUT, stops issuing,
// waits (bounded) for its MMAs and frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "pc_internal.cuh"

namespace {

constexpr int kChunk = 16;
constexpr long kSpinLimit = 1L << 26;


__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int kmaj_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets, fixed version bits 46-48 = 0b001, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// Two floats split into packed (hi, lo) pairs of the operand type.
template <int kBf16>
__device__ __forceinline__ void split2(float x, float y, uint32_t* hi, uint32_t* lo) {
  if (kBf16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    *hi = *reinterpret_cast<const uint32_t*>(&h);
    *lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __half2 h = __floats2half2_rn(x, y);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(x - hf.x, y - hf.y);
    *hi = *reinterpret_cast<const uint32_t*>(&h);
    *lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}

// 16 values (one per particle of the chunk) of one operand row, hi part to row
// `row` and lo part to row `row + lo_off`.
template <int kBf16>
__device__ __forceinline__ void store_row(uint8_t* tile, int row, int lo_off, const float v[16]) {
  uint32_t hi[8], lo[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) split2<kBf16>(v[2 * q], v[2 * q + 1], &hi[q], &lo[q]);
  *reinterpret_cast<uint4*>(tile + kmaj_off(row, 0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(tile + kmaj_off(row, 8)) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
  *reinterpret_cast<uint4*>(tile + kmaj_off(row + lo_off, 0)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  *reinterpret_cast<uint4*>(tile + kmaj_off(row + lo_off, 8)) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
}

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float r[64]) {
  uint32_t u[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
        "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
        "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31]),
        "=r"(u[32]), "=r"(u[33]), "=r"(u[34]), "=r"(u[35]), "=r"(u[36]), "=r"(u[37]), "=r"(u[38]), "=r"(u[39]),
        "=r"(u[40]), "=r"(u[41]), "=r"(u[42]), "=r"(u[43]), "=r"(u[44]), "=r"(u[45]), "=r"(u[46]), "=r"(u[47]),
        "=r"(u[48]), "=r"(u[49]), "=r"(u[50]), "=r"(u[51]), "=r"(u[52]), "=r"(u[53]), "=r"(u[54]), "=r"(u[55]),
        "=r"(u[56]), "=r"(u[57]), "=r"(u[58]), "=r"(u[59]), "=r"(u[60]), "=r"(u[61]), "=r"(u[62]), "=r"(u[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 64; ++c) r[c] = __uint_as_float(u[c]);
}

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

constexpr int kProducers = 8;                           // producer warps, one TMEM accumulator each
constexpr int kEpiWarps = 4;                            // one per TMEM lane quarter
constexpr int kThreads2 = 32 * (kProducers + kEpiWarps + 1);
constexpr int kRing = 2;                                // operand slots per producer
constexpr int kList = 64;                               // kept-particle ring (>= kChunk + 32)
constexpr int kQ = 16;                                  // finished-element queue (>= 2 kProducers)

struct __align__(1024) TcSmem2 {
  uint8_t a[kProducers][kRing][4096];
  uint8_t b[kProducers][kRing][2048];
  float pf[kProducers][kChunk][28];
  float4 lrec[kProducers][kList][4];  // the kept particles' records
  int lmeta[kProducers][kList];
  float comb[64][33];
  int pre[kProducers][128];
  int rbeg[kProducers][128];
  int meta[kProducers][kRing][4];  // element, accumulate flag, last-chunk flag
  unsigned long long full[kProducers][kRing];
  unsigned long long empty[kProducers][kRing];
  unsigned long long acc_full[kProducers];
  unsigned long long acc_empty[kProducers];  // 2 arrivals: epilogue quarters 0 and 1
  unsigned long long comb_full;              // 2 arrivals: epilogue quarters 2 and 3
  unsigned long long comb_empty;             // 2 arrivals: epilogue quarters 0 and 1
  unsigned long long fin;
  int qe[kQ];
  int qb[kQ];
  int q_tail;
  int prod_total[kProducers];
  int failed;
  uint32_t tmem_base;
};

__device__ __forceinline__ int vload(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ void vstore(int* p, int v) { *(volatile int*)p = v; }

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

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fail_now(TcSmem2& S, unsigned long long* counters) {
  vstore(&S.failed, 1);
  atomicMax(counters, (unsigned long long)PC_ETIMEOUT);
}

// Producer warp w: owns elements blockIdx.x * kProducers + w + k * gridDim.x * kProducers.
// Per element: neighbour ranges, ordered warp-level compaction of the particles
// whose support reaches the element, then per 16 kept particles: factors (lane
// parallel), the operand rows (3 per lane) into its ring slot, and a release
// arrival on the slot's full barrier for the MMA thread.
template <int kBf16>
__device__ void tc_producer(TcSmem2& S, const TcDepositArgs& A, int w, int lane) {
  const int n1 = A.n1, ne = A.ne, rho = A.rho, span = 2 * rho + 1, nrange = span * span * span;
  const int nodes = n1 * n1 * n1;
  const int64_t nel = (int64_t)ne * ne * ne;
  int chunk = 0;
  for (int64_t e = (int64_t)blockIdx.x * kProducers + w; e < nel; e += (int64_t)gridDim.x * kProducers) {
    if (vload(&S.failed)) break;
    const int ex = (int)(e % ne), ey = (int)((e / ne) % ne), ez = (int)(e / ((int64_t)ne * ne));
    for (int r = lane; r < nrange; r += 32) {
      const int dx = r % span - rho, dy = (r / span) % span - rho, dz = r / (span * span) - rho;
      const int nb = (wrapi(ez + dz, ne) * ne + wrapi(ey + dy, ne)) * ne + wrapi(ex + dx, ne);
      const int b0 = A.start[nb], b1 = A.start[nb + 1];
      S.rbeg[w][r] = b0;
      S.pre[w][r + 1] = b1 - b0;
    }
    __syncwarp();
    if (lane == 0) {
      S.pre[w][0] = 0;
      for (int r = 1; r <= nrange; ++r) S.pre[w][r] += S.pre[w][r - 1];
    }
    __syncwarp();
    const int total = S.pre[w][nrange];
    int nmma = 0;
    int scan = 0;
    int head = 0, tail = 0;  // kept-particle ring: [head, tail)
    // candidate batch [scan, scan + 32) loaded one batch ahead, so that its global
    // load latency overlaps the previous chunk's work
    float4 c0r, c1r, c2r, c3r;
    int cmeta = 0;
    bool cvalid = false;
    auto load_batch = [&](int base) {
      const int idx = base + lane;
      cvalid = idx < total;
      if (cvalid) {
        int r = 0;
        while (S.pre[w][r + 1] <= idx) ++r;
        const int64_t j = S.rbeg[w][r] + (idx - S.pre[w][r]);
        const int d3[3] = {r % span - rho, (r / span) % span - rho, r / (span * span) - rho};
        cmeta = (rho - d3[0]) | ((rho - d3[1]) << 4) | ((rho - d3[2]) << 8);
        c0r = A.rec[4 * j];
        c1r = A.rec[4 * j + 1];
        c2r = A.rec[4 * j + 2];
        c3r = A.rec[4 * j + 3];
      }
    };
    if (total > 0) load_batch(0);
    for (;;) {
      // refill until the ring holds more than one chunk or the neighbourhood is exhausted,
      // so that "last chunk of the element" is known exactly
      while (scan < total && tail - head <= kChunk) {
        bool keep = false;
        if (cvalid) {
          const unsigned mk[3] = {__float_as_uint(c2r.z), __float_as_uint(c2r.w), __float_as_uint(c3r.x)};
          keep = true;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int wo = (cmeta >> (4 * a)) & 15;
            keep = keep && ((mk[a] >> (wo * n1)) & ((1u << n1) - 1u)) != 0u;
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          const int pos = (tail + __popc(bal & ((1u << lane) - 1u))) & (kList - 1);
          S.lrec[w][pos][0] = c0r;
          S.lrec[w][pos][1] = c1r;
          S.lrec[w][pos][2] = c2r;
          S.lrec[w][pos][3] = c3r;
          S.lmeta[w][pos] = cmeta;
        }
        tail += __popc(bal);
        scan += 32;
        if (scan < total) load_batch(scan);
      }
      __syncwarp();
      const int avail = tail - head;
      if (avail == 0) break;
      const int take = avail < kChunk ? avail : kChunk;
      const bool last = avail <= kChunk;  // the refill stopped short only because the scan is done
      const int slot = chunk % kRing;
      if (chunk >= kRing) {
        const uint32_t par = (uint32_t)((chunk / kRing - 1) & 1);
        long it = 0;
        while (!mbar_try(&S.empty[w][slot], par)) {
          if (++it > kSpinLimit || vload(&S.failed)) {
            if (lane == 0) fail_now(S, A.counters + CNT_STATUS);
            return;
          }
        }
      }
      // factors: lane -> particle p = lane & 15, values 12 h .. 12 h + 11 of (kx[8] ky[8] kz[8])
      {
        const int p = lane & 15, hlf = lane >> 4;
        float* pf = S.pf[w][p];
        if (p < take) {
          const int pos = (head + p) & (kList - 1);
          const int meta = S.lmeta[w][pos];
          const float4 r0 = S.lrec[w][pos][0], r1 = S.lrec[w][pos][1], r2 = S.lrec[w][pos][2], r3 = S.lrec[w][pos][3];
          const float t3[3] = {r0.x, r0.y, r0.z}, iz[3] = {r0.w, r1.x, r1.y};
          const unsigned mk[3] = {__float_as_uint(r2.z), __float_as_uint(r2.w), __float_as_uint(r3.x)};
#pragma unroll
          for (int u = 0; u < 12; ++u) {
            const int v = 12 * hlf + u, a = v >> 3, i = v & 7;
            float f = 0.0f;
            if (i < n1) {
              const int wo = (meta >> (4 * a)) & 15;
              if ((mk[a] >> (wo * n1 + i)) & 1u) {
                const float d = (float)(wo - rho) + A.s[i] - t3[a];
                f = exp2f(-(d * d) * A.c2l) * iz[a];
              }
            }
            pf[v] = f;
          }
          if (hlf == 0) {
            pf[24] = r1.z;
            pf[25] = r1.w;
            pf[26] = r2.x;
            pf[27] = r2.y;
          }
        } else {
#pragma unroll
          for (int u = 0; u < 12; ++u) pf[12 * hlf + u] = 0.0f;
          if (hlf == 0) pf[24] = pf[25] = pf[26] = pf[27] = 0.0f;
        }
      }
      __syncwarp();
      // operand rows: 0..63 YZ (A operand, hi + lo), 64..95 q kx (B operand, hi + lo)
#pragma unroll
      for (int rr = 0; rr < 3; ++rr) {
        const int row = lane + 32 * rr;
        float v[16];
        if (row < 64) {
          if (row < n1 * n1) {
            const int jj = row % n1, kk = row / n1;
#pragma unroll
            for (int p = 0; p < kChunk; ++p) v[p] = S.pf[w][p][8 + jj] * S.pf[w][p][16 + kk] * 256.0f;
            store_row<kBf16>(S.a[w][slot], row, 64, v);
          }
        } else {
          const int ci = row - 64;
          if (ci < 4 * n1) {
            const int c = ci / n1, i = ci % n1;
#pragma unroll
            for (int p = 0; p < kChunk; ++p) v[p] = S.pf[w][p][24 + c] * S.pf[w][p][i] * 16.0f;
            store_row<kBf16>(S.b[w][slot], ci, 32, v);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        S.meta[w][slot][0] = (int)e;
        S.meta[w][slot][1] = nmma > 0 ? 1 : 0;
        S.meta[w][slot][2] = last ? 1 : 0;
        mbar_arrive(&S.full[w][slot]);
      }
      head += take;
      ++nmma;
      ++chunk;
      if (last) break;
    }
    if (nmma == 0) {
      float* out = A.field + e * 4 * nodes;
      for (int a = lane; a < 4 * nodes; a += 32) out[a] = 0.0f;
    }
  }
  __syncwarp();
  if (lane == 0) {
    __threadfence_block();
    vstore(&S.prod_total[w], chunk);
  }
}

// The MMA thread: serves the producers' rings in turn; before the first chunk of a
// producer's element it waits (without blocking the others) for the epilogue to
// have emptied that producer's accumulator; after an element's last chunk it commits
// the accumulator and queues (element, producer) for the epilogue.
__device__ void tc_mma(TcSmem2& S, const TcDepositArgs& A, uint32_t tmem, uint32_t idesc) {
  int used[kProducers], eng[kProducers];
  for (int w = 0; w < kProducers; ++w) used[w] = eng[w] = 0;
  int qt = 0;
  long idle = 0;
  for (;;) {
    if (vload(&S.failed)) break;
    bool all_done = true, progress = false;
    for (int w = 0; w < kProducers; ++w) {
      const int tot = vload(&S.prod_total[w]);
      if (tot >= 0 && eng[w] >= tot) continue;
      all_done = false;
      const int c = eng[w], slot = c % kRing;
      if (!mbar_try(&S.full[w][slot], (uint32_t)((c / kRing) & 1))) continue;
      const int e = S.meta[w][slot][0], acc = S.meta[w][slot][1], last = S.meta[w][slot][2];
      if (!acc) {
        if (used[w] >= 1 && !mbar_try(&S.acc_empty[w], (uint32_t)((used[w] - 1) & 1))) continue;
        ++used[w];
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      mma_issue(tmem + 64u * w, make_desc(smem_u32(S.a[w][slot]), 128, 256), make_desc(smem_u32(S.b[w][slot]), 128, 256),
                idesc, (uint32_t)acc);
      mma_commit(&S.empty[w][slot]);
      if (last) {
        mma_commit(&S.acc_full[w]);
        S.qe[qt % kQ] = e;
        S.qb[qt % kQ] = w;
        __threadfence_block();
        vstore(&S.q_tail, ++qt);
      }
      ++eng[w];
      progress = true;
    }
    if (all_done) break;
    if (progress) {
      idle = 0;
    } else if (++idle > kSpinLimit) {
      fail_now(S, A.counters + CNT_STATUS);
      break;
    }
  }
  // every MMA issued so far has completed once this commit arrives
  mma_commit(&S.fin);
  (void)mbar_wait(&S.fin, 0);
  S.qe[qt % kQ] = -1;
  S.qb[qt % kQ] = 0;
  __threadfence_block();
  vstore(&S.q_tail, ++qt);
}

// Epilogue warp for TMEM lane quarter q: drains the finished-element queue in order.
__device__ void tc_epilogue(TcSmem2& S, const TcDepositArgs& A, uint32_t tmem, int q, int lane) {
  const int n1 = A.n1, nodes = n1 * n1 * n1;
  int seen[kProducers];
  for (int w = 0; w < kProducers; ++w) seen[w] = 0;
  for (int k = 0;; ++k) {
    long it = 0;
    while (vload(&S.q_tail) <= k) {
      if (++it > kSpinLimit || vload(&S.failed)) {
        if (lane == 0 && q == 0 && !vload(&S.failed)) fail_now(S, A.counters + CNT_STATUS);
        return;
      }
    }
    const int e = vload(&S.qe[k % kQ]), w = vload(&S.qb[k % kQ]);
    if (e < 0) return;
    if (!mbar_wait(&S.acc_full[w], (uint32_t)(seen[w] & 1))) {
      if (lane == 0) fail_now(S, A.counters + CNT_STATUS);
      return;
    }
    ++seen[w];
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float r[64];
    tmem_ld64(tmem + 64u * w + ((uint32_t)(32 * q) << 16), r);
    const int jk = 32 * (q & 1) + lane;
    if (q >= 2) {
      // rows 64..127 (YZ lo): add the two column halves into comb for quarters 0 and 1
      if (k >= 1 && !mbar_wait(&S.comb_empty, (uint32_t)((k - 1) & 1))) {
        if (lane == 0) fail_now(S, A.counters + CNT_STATUS);
        return;
      }
#pragma unroll
      for (int ci = 0; ci < 32; ++ci) S.comb[jk][ci] = r[ci] + r[32 + ci];
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.comb_full);
    } else {
      if (!mbar_wait(&S.comb_full, (uint32_t)(k & 1))) {
        if (lane == 0) fail_now(S, A.counters + CNT_STATUS);
        return;
      }
      if (jk < n1 * n1) {
        float* out = A.field + (int64_t)e * 4 * nodes;
        for (int ci = 0; ci < 4 * n1; ++ci) {
          const int c = ci / n1, i = ci % n1;
          out[c * nodes + jk * n1 + i] = ((r[ci] + r[32 + ci]) + S.comb[jk][ci]) * A.scale_out;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&S.comb_empty);
        // quarters 2 and 3 finished their loads before comb_full; 0 and 1 arrive here
        mbar_arrive(&S.acc_empty[w]);
      }
    }
  }
}

template <int kBf16>
__global__ void __launch_bounds__(kThreads2, 1) k_tc_deposit(TcDepositArgs A) {
  extern __shared__ uint8_t smraw[];
  TcSmem2& S = *reinterpret_cast<TcSmem2*>(smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < kProducers * kRing * 4096 / 16; i += kThreads2)
    reinterpret_cast<uint4*>(&S.a[0][0][0])[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < kProducers * kRing * 2048 / 16; i += kThreads2)
    reinterpret_cast<uint4*>(&S.b[0][0][0])[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int w = 0; w < kProducers; ++w) {
      for (int s = 0; s < kRing; ++s) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.full[w][s])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.empty[w][s])));
      }
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.acc_full[w])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(smem_u32(&S.acc_empty[w])));
      S.prod_total[w] = -1;
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.fin)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(smem_u32(&S.comb_full)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(smem_u32(&S.comb_empty)));
    S.q_tail = 0;
    S.failed = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(64u * kProducers));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem_base;
  const uint32_t fmt = kBf16 ? 1u : 0u;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (8u << 17) | (8u << 24);
  if (warp < kProducers) {
    tc_producer<kBf16>(S, A, warp, lane);
  } else if (warp < kProducers + kEpiWarps) {
    tc_epilogue(S, A, tmem, warp - kProducers, lane);
  } else if (lane == 0) {
    tc_mma(S, A, tmem, idesc);
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64u * kProducers));
}

}  // namespace

cudaError_t pc_tc_deposit_launch(const TcDepositArgs& A, cudaStream_t st, int* nblocks) {
  const size_t smem = sizeof(TcSmem2) + 1024;
  const int64_t nel = (int64_t)A.ne * A.ne * A.ne;
  int dev = 0, sms = 0;
  PC_CUDA_TRY(cudaGetDevice(&dev));
  PC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // one persistent CTA per SM: it holds all 512 tensor-memory columns
  int64_t grid = (nel + kProducers - 1) / kProducers;
  if (grid > sms) grid = sms;
  if (grid < 1) grid = 1;
  *nblocks = (int)grid;
  if (A.tc_type == PC_TC_BF16) {
    PC_CUDA_TRY(cudaFuncSetAttribute(k_tc_deposit<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_deposit<1><<<(unsigned)grid, kThreads2, smem, st>>>(A);
  } else {
    PC_CUDA_TRY(cudaFuncSetAttribute(k_tc_deposit<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_deposit<0><<<(unsigned)grid, kThreads2, smem, st>>>(A);
  }
  return cudaGetLastError();
}
