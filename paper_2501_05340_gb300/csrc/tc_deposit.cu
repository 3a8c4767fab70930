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
// Each of the 8 producer warps owns one 64-column accumulator in tensor memory and
// builds, for one element at a time, the operand tiles of 16 kept particles; its
// lane 0 issues the tcgen05.mma and a tcgen05.commit that arrives on the slot's
// mbarrier when the tensor core has read it (commits track the issuing thread's own
// MMAs, so producers need no common issuer). After an element's last chunk the
// producer queues (element, producer); 4 epilogue warps, one per TMEM lane quarter,
// drain the queue. Every wait is bounded in wall-clock time: on expiry the kernel
// records PC_ETIMEOUT, stops issuing, waits (bounded) for its MMAs and frees its
// tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "pc_internal.cuh"

namespace {

constexpr int kChunk = 16;


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

constexpr int kProducers = 8;                       // producer warps, one TMEM accumulator each
constexpr int kEpiWarps = 4;                        // one per TMEM lane quarter
constexpr int kThreads = 32 * (kProducers + kEpiWarps);
constexpr int kRing = 2;                            // operand slots per producer
constexpr int kList = 64;                           // kept-particle ring (>= kChunk + 32)
constexpr int kQ = 32;                              // finished-element queue (>= 2 kProducers)
constexpr int kMaxRanges = 125;                     // (2 rho + 1)^3 neighbour cells, rho <= 2
constexpr int kPf = 20;                             // words per factor row: 16 particles + pad
constexpr unsigned long long kWaitNs = 2000000000;  // a wait without progress for 2 s fails

// Per-producer factor rows are [v][p] with v = 8 a + i (axis a, node i) and 24 + c
// (charge c); the row pitch of 20 words keeps both the lane-per-particle stores and
// the float4 row reads free of bank conflicts. Kept records are stored as four
// planes of float4 so that consecutive ring positions hit consecutive banks.
struct __align__(1024) TcSmem {
  uint8_t a[kProducers][kRing][4096];
  uint8_t b[kProducers][kRing][2048];
  float pf[kProducers][28][kPf];
  float4 lrec[kProducers][4][kList];
  int lmeta[kProducers][kList];
  float comb[64][33];
  int pre[kProducers][kMaxRanges + 1];
  int rbeg[kProducers][kMaxRanges];
  int rmeta[kProducers][kMaxRanges];
  unsigned long long empty[kProducers][kRing];  // tcgen05.commit: the slot has been read
  unsigned long long acc_full[kProducers];      // tcgen05.commit: the element's MMAs are done
  unsigned long long acc_empty[kProducers];     // 2 arrivals: epilogue quarters 0 and 1
  unsigned long long fin[kProducers];           // tcgen05.commit at producer exit
  unsigned long long qfull[kQ];                 // queue entry written
  unsigned long long comb_full;                 // 2 arrivals: epilogue quarters 2 and 3
  unsigned long long comb_empty;                // 2 arrivals: epilogue quarters 0 and 1
  int qe[kQ];
  int qb[kQ];
  int q_head;
  int progress[kProducers];
  int failed;
  uint32_t tmem_base;
};

__device__ __forceinline__ int vload(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ void vstore(int* p, int v) { *(volatile int*)p = v; }

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

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

// Waits for the phase of the given parity. Returns false once the block has failed,
// or after kWaitNs without completion.
__device__ bool mbar_wait(unsigned long long* bar, uint32_t parity, const int* failed) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63u) == 0u && (vload(failed) || gtime() - t0 > kWaitNs)) return false;
  }
}

__device__ __forceinline__ void fail_now(TcSmem& S, unsigned long long* counters) {
  vstore(&S.failed, 1);
  atomicMax(counters, (unsigned long long)PC_ETIMEOUT);
}

// Queue push by a producer's lane 0: (element, producer) or the exit sentinel e = -1.
__device__ __forceinline__ void queue_push(TcSmem& S, int e, int w) {
  const int k = atomicAdd(&S.q_head, 1);
  S.qe[k % kQ] = e;
  S.qb[k % kQ] = w;
  mbar_arrive(&S.qfull[k % kQ]);  // release: the entry is visible to the waiter
}

// Producer warp w: owns elements blockIdx.x * kProducers + w + k * gridDim.x * kProducers.
// Per element: the (2 rho + 1)^3 neighbour cell ranges and their prefix sum, ordered
// warp-level compaction of the particles whose support reaches the element, then per
// 16 kept particles: factors (lane parallel), the operand rows (3 per lane) into a
// ring slot, and one tcgen05.mma into the producer's own accumulator, issued by
// lane 0. Accumulation order inside an element is the kept order, so the deposit is
// deterministic.
template <int kBf16>
__device__ void tc_producer(TcSmem& S, const TcDepositArgs& A, uint32_t tmem, uint32_t idesc, int w, int lane) {
  const int n1 = A.n1, ne = A.ne, rho = A.rho, span = 2 * rho + 1, nrange = span * span * span;
  const int nodes = n1 * n1 * n1;
  const int64_t nel = (int64_t)ne * ne * ne;
  int top = 1;
  while (2 * top < nrange) top *= 2;
  // factor slots of this lane: particle p, nodes 4 hh .. 4 hh + 3 of each axis
  const int p = lane & 15, hh = lane >> 4;
  const unsigned lanemask = (((1u << n1) - 1u) >> (4 * hh)) & 15u;
  float sv[4];
#pragma unroll
  for (int ii = 0; ii < 4; ++ii) sv[ii] = (4 * hh + ii < n1) ? A.s[4 * hh + ii] : 0.0f;
  const float c2l = A.c2l;
  const uint32_t acc = tmem + 64u * (uint32_t)w;
  int chunk = 0, used = 0;
  bool ok = true;
  for (int64_t e = (int64_t)blockIdx.x * kProducers + w; ok && e < nel; e += (int64_t)gridDim.x * kProducers) {
    if (__any_sync(0xffffffffu, vload(&S.failed))) break;
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
        S.rbeg[w][r] = b0;
        S.rmeta[w][r] = (rho - dx) | ((rho - dy) << 4) | ((rho - dz) << 8);
      }
      int x = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (r < nrange) S.pre[w][r + 1] = total + x;
      total += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) S.pre[w][0] = 0;
    __syncwarp();
    int nmma = 0, scan = 0, head = 0, tail = 0;  // kept-particle ring: [head, tail)
    // candidate batch [scan, scan + 32), loaded one batch ahead
    float4 c0r, c1r, c2r, c3r;
    int cmeta = 0;
    bool cvalid = false;
    auto load_batch = [&](int base) {
      const int idx = base + lane;
      cvalid = idx < total;
      if (cvalid) {
        int r = 0;
        for (int stp = top; stp > 0; stp >>= 1)
          if (r + stp < nrange && S.pre[w][r + stp] <= idx) r += stp;
        cmeta = S.rmeta[w][r];
        const int64_t j = (int64_t)S.rbeg[w][r] + (idx - S.pre[w][r]);
        c0r = A.rec[4 * j];
        c1r = A.rec[4 * j + 1];
        c2r = A.rec[4 * j + 2];
        c3r = A.rec[4 * j + 3];
      }
    };
    if (total > 0) load_batch(0);
    for (;;) {
      // refill until the ring holds more than one chunk or the neighbourhood is
      // exhausted, so that "last chunk of the element" is known exactly
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
          S.lrec[w][0][pos] = c0r;
          S.lrec[w][1][pos] = c1r;
          S.lrec[w][2][pos] = c2r;
          S.lrec[w][3][pos] = c3r;
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
      // factors into pf: lane -> particle p, nodes 4 hh + ii; kx scaled by 2^4, kz by 2^8
      {
        float f[3][4] = {};
        float qv[2] = {0.0f, 0.0f};
        if (p < take) {
          const int pos = (head + p) & (kList - 1);
          const int meta = S.lmeta[w][pos];
          const float4 r0 = S.lrec[w][0][pos], r1 = S.lrec[w][1][pos], r2 = S.lrec[w][2][pos], r3 = S.lrec[w][3][pos];
          const float t3[3] = {r0.x, r0.y, r0.z};
          const float iz[3] = {r0.w * 16.0f, r1.x, r1.y * 256.0f};
          const unsigned mk[3] = {__float_as_uint(r2.z), __float_as_uint(r2.w), __float_as_uint(r3.x)};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int wo = (meta >> (4 * a)) & 15;
            const int sh = wo * n1 + 4 * hh;
            const unsigned bits = (sh < 32 ? (mk[a] >> sh) : 0u) & lanemask;
            const float base = (float)(wo - rho) - t3[a];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) {
              const float d = base + sv[ii];
              const float g = exp2f(-(d * d) * c2l) * iz[a];
              f[a][ii] = ((bits >> ii) & 1u) ? g : 0.0f;
            }
          }
          qv[0] = hh ? r2.x : r1.z;
          qv[1] = hh ? r2.y : r1.w;
        }
        float* pf = &S.pf[w][0][0];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) pf[(8 * a + 4 * hh + ii) * kPf + p] = f[a][ii];
        pf[(24 + 2 * hh) * kPf + p] = qv[0];
        pf[(25 + 2 * hh) * kPf + p] = qv[1];
      }
      const int slot = chunk % kRing;
      const bool free_slot =
          chunk < kRing || mbar_wait(&S.empty[w][slot], (uint32_t)((chunk / kRing - 1) & 1), &S.failed);
      if (!__all_sync(0xffffffffu, free_slot)) {
        if (lane == 0) fail_now(S, A.counters + CNT_STATUS);
        ok = false;
        break;
      }
      __syncwarp();
      // operand rows: lane and lane + 32 of YZ (A operand), lane of q kx (B operand)
#pragma unroll
      for (int rr = 0; rr < 3; ++rr) {
        const int row = lane + 32 * rr;
        const bool is_a = rr < 2;
        const int nrows = is_a ? n1 * n1 : 4 * n1;
        const int lr = is_a ? row : lane;
        if (lr < nrows) {
          const int u0 = is_a ? 8 + lr % n1 : 24 + lr / n1;  // ky_j  or q_c
          const int u1 = is_a ? 16 + lr / n1 : lr % n1;      // kz_k  or kx_i
          const float4* x0 = reinterpret_cast<const float4*>(&S.pf[w][u0][0]);
          const float4* x1 = reinterpret_cast<const float4*>(&S.pf[w][u1][0]);
          float v[16];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const float4 g = x0[t], h = x1[t];
            v[4 * t] = g.x * h.x;
            v[4 * t + 1] = g.y * h.y;
            v[4 * t + 2] = g.z * h.z;
            v[4 * t + 3] = g.w * h.w;
          }
          if (is_a)
            store_row<kBf16>(S.a[w][slot], lr, 64, v);
          else
            store_row<kBf16>(S.b[w][slot], lr, 32, v);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        bool go = true;
        if (nmma == 0 && used > 0)  // the epilogue has read this accumulator's previous element
          go = mbar_wait(&S.acc_empty[w], (uint32_t)((used - 1) & 1), &S.failed);
        if (go) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          mma_issue(acc, make_desc(smem_u32(S.a[w][slot]), 128, 256), make_desc(smem_u32(S.b[w][slot]), 128, 256),
                    idesc, nmma > 0 ? 1u : 0u);
          mma_commit(&S.empty[w][slot]);
          if (last) {
            mma_commit(&S.acc_full[w]);
            queue_push(S, (int)e, w);
          }
          vstore(&S.progress[w], chunk + 1);
        } else {
          fail_now(S, A.counters + CNT_STATUS);
        }
      }
      if (__shfl_sync(0xffffffffu, vload(&S.failed), 0)) {
        ok = false;
        break;
      }
      if (nmma == 0) ++used;
      head += take;
      ++nmma;
      ++chunk;
      if (last) break;
    }
    if (ok && nmma == 0) {
      float* out = A.field + e * 4 * nodes;
      for (int k = lane; k < 4 * nodes; k += 32) out[k] = 0.0f;
    }
  }
  __syncwarp();
  if (lane == 0) {
    // every MMA this thread issued has completed once this commit arrives
    mma_commit(&S.fin[w]);
    int never = 0;
    (void)mbar_wait(&S.fin[w], 0, &never);
    queue_push(S, -1, w);
  }
}

// Epilogue warp for TMEM lane quarter q: drains the finished-element queue in
// order until every producer has sent its exit sentinel.
__device__ void tc_epilogue(TcSmem& S, const TcDepositArgs& A, uint32_t tmem, int q, int lane) {
  const int n1 = A.n1, nodes = n1 * n1 * n1;
  unsigned seen = 0u;  // bit w: parity of the next acc_full phase of producer w
  int exited = 0;
  for (int k = 0; exited < kProducers; ++k) {
    // the next entry may be a whole element away: time out only without producer progress
    {
      unsigned long long t0 = gtime();
      int last_sum = -1;
      for (unsigned it = 0; !mbar_try(&S.qfull[k % kQ], (uint32_t)((k / kQ) & 1)); ++it) {
        if ((it & 63u) != 63u) continue;
        if (vload(&S.failed)) return;
        const unsigned long long now = gtime();
        if (now - t0 > kWaitNs) {
          int sum = 0;
          for (int w = 0; w < kProducers; ++w) sum += vload(&S.progress[w]);
          if (sum == last_sum) {
            if (lane == 0 && q == 0) fail_now(S, A.counters + CNT_STATUS);
            return;
          }
          last_sum = sum;
          t0 = now;
        }
      }
    }
    const int e = vload(&S.qe[k % kQ]), w = vload(&S.qb[k % kQ]);
    if (e < 0) {
      ++exited;
      continue;
    }
    if (!mbar_wait(&S.acc_full[w], (seen >> w) & 1u, &S.failed)) {
      if (lane == 0) fail_now(S, A.counters + CNT_STATUS);
      return;
    }
    seen ^= 1u << w;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float r[64];
    tmem_ld64(tmem + 64u * w + ((uint32_t)(32 * q) << 16), r);
    const int jk = 32 * (q & 1) + lane;
    const int m = k - exited;  // index of this element among the drained ones
    if (q >= 2) {
      // rows 64..127 (YZ lo): add the two column halves into comb for quarters 0 and 1
      if (m >= 1 && !mbar_wait(&S.comb_empty, (uint32_t)((m - 1) & 1), &S.failed)) {
        if (lane == 0) fail_now(S, A.counters + CNT_STATUS);
        return;
      }
#pragma unroll
      for (int ci = 0; ci < 32; ++ci) S.comb[jk][ci] = r[ci] + r[32 + ci];
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.comb_full);
    } else {
      if (!mbar_wait(&S.comb_full, (uint32_t)(m & 1), &S.failed)) {
        if (lane == 0) fail_now(S, A.counters + CNT_STATUS);
        return;
      }
      if (jk < n1 * n1) {
        float* out = A.field + (int64_t)e * 4 * nodes;
#pragma unroll
        for (int ci = 0; ci < 32; ++ci) {
          if (ci < 4 * n1) {
            const int c = ci / n1, i = ci - c * n1;
            out[c * nodes + jk * n1 + i] = ((r[ci] + r[32 + ci]) + S.comb[jk][ci]) * A.scale_out;
          }
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
__global__ void __launch_bounds__(kThreads, 1) k_tc_deposit(TcDepositArgs A) {
  extern __shared__ uint8_t smraw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < kProducers * kRing * 4096 / 16; i += kThreads)
    reinterpret_cast<uint4*>(&S.a[0][0][0])[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < kProducers * kRing * 2048 / 16; i += kThreads)
    reinterpret_cast<uint4*>(&S.b[0][0][0])[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int w = 0; w < kProducers; ++w) {
      for (int s = 0; s < kRing; ++s)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.empty[w][s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.acc_full[w])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(smem_u32(&S.acc_empty[w])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.fin[w])));
      S.progress[w] = 0;
    }
    for (int k = 0; k < kQ; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.qfull[k])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(smem_u32(&S.comb_full)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(smem_u32(&S.comb_empty)));
    S.q_head = 0;
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
  if (warp < kProducers)
    tc_producer<kBf16>(S, A, tmem, idesc, warp, lane);
  else
    tc_epilogue(S, A, tmem, warp - kProducers, lane);
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64u * kProducers));
}

}  // namespace

cudaError_t pc_tc_deposit_launch(const TcDepositArgs& A, cudaStream_t st, int* nblocks) {
  const size_t smem = sizeof(TcSmem) + 1024;
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
    k_tc_deposit<1><<<(unsigned)grid, kThreads, smem, st>>>(A);
  } else {
    PC_CUDA_TRY(cudaFuncSetAttribute(k_tc_deposit<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_deposit<0><<<(unsigned)grid, kThreads, smem, st>>>(A);
  }
  return cudaGetLastError();
}
