// Tensor-core deposit of the mixed-precision projection (tcgen05, sm_103a).
//
// For one element with n1 = N+1 <= 8 Gauss nodes per axis the separable deposit is
//   D[jk][c i] = sum_p YZ[p][jk] A[p][c i],  YZ = ky_j kz_k,  A = q_c kx_i,
// a dense contraction over the particles p whose support reaches the element.
// Each factor is split into a high and a low part of the operand type (FP16 or
// BF16) and one MMA of M = 128, N = 64, K = 16 computes all four products at once:
//   A operand row 32 q + r: YZ_hi of jk = 16 q + r, row 32 q + 16 + r: its YZ_lo
//     (q = 0..3, r = 0..15; YZ scaled by 2^8)
//   B operand rows  0..31 : A_hi  (scaled by 2^4), rows 32..63 : A_lo
// so D holds, in every tensor-memory lane quarter, the products hi hi, hi lo, lo hi
// and lo lo of 16 rows jk, and the element's deposit is their sum (the lo*lo one is
// below the accuracy of the others and harmless). An epilogue warp reads its own
// quarter and adds the lo rows to the hi rows with one shuffle.
//
// Operands live in shared memory in the MN-major layout without swizzle: core
// matrices of 8 particles (K) x 16 bytes (8 consecutive rows of M or N), the row
// groups 128 B apart and the particle octets one row-group column apart (2048 B for
// A, 1024 B for B). So one lane per particle writes its own 16-byte pieces: no
// factor tile is staged, and every store is a whole core-matrix row.
// Each of 8 worker warps owns one 64-column accumulator in tensor memory and works on
// one element at a time: it compacts the particles that reach the element into a
// ring (order kept), and per 32 of them every lane computes its particle's factors
// in registers and writes the operands into the worker's stage; lane 0
// issues the two MMAs (K = 16 each) and a tcgen05.commit that arrives on the stage's
// mbarrier when the tensor core has read it. After an element's last chunk the
// worker queues (element, worker); 4 epilogue warps, one per TMEM lane quarter,
// drain the queue. Every wait is bounded in wall-clock time: on expiry the kernel
// records PC_ETIMEOUT, stops issuing, waits (bounded) for its MMAs and frees its
// tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "pc_internal.cuh"

namespace {



__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

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
    const float2 r = __fadd2_rn(make_float2(x, y), make_float2(-hf.x, -hf.y));
    const __nv_bfloat162 l = __floats2bfloat162_rn(r.x, r.y);
    *hi = *reinterpret_cast<const uint32_t*>(&h);
    *lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __half2 h = __floats2half2_rn(x, y);
    const float2 hf = __half22float2(h);
    const float2 r = __fadd2_rn(make_float2(x, y), make_float2(-hf.x, -hf.y));
    const __half2 l = __floats2half2_rn(r.x, r.y);
    *hi = *reinterpret_cast<const uint32_t*>(&h);
    *lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

constexpr int kChunk = 32;                          // particles per operand stage (two MMAs)
constexpr int kWorkers = 8;                         // worker warps, one TMEM accumulator each (all 512 columns)
constexpr int kEpiWarps = 4;                        // one per TMEM lane quarter
constexpr int kThreads = 32 * (kWorkers + kEpiWarps);
constexpr int kStages = 1;                          // operand stages per worker (a chunk's MMAs finish while
                                                    // the worker compacts and builds the next)
constexpr int kList = 64;                           // kept-particle ring (>= kChunk + 32)
constexpr int kQ = 32;                              // finished-element queue (>= 2 kWorkers)
constexpr int kMaxRanges = 125;                     // (2 rho + 1)^3 neighbour cells, rho <= 2
constexpr int kAStage = 8192;                       // A: 128 rows x 32 particles x 2 B
constexpr int kBStage = 4096;                       // B: 64 rows x 32 particles x 2 B
constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kWaitNs = 2000000000;  // a wait without progress for 2 s fails

// Kept records are stored as four planes of float4 so that consecutive ring
// positions hit consecutive banks.
struct __align__(1024) TcSmem {
  uint8_t a[kWorkers][kStages][kAStage];
  uint8_t b[kWorkers][kStages][kBStage];
  float4 lrec[kWorkers][4][kList];
  int lmeta[kWorkers][kList];
  int pre[kWorkers][kMaxRanges + 1];
  int rbeg[kWorkers][kMaxRanges];
  int rmeta[kWorkers][kMaxRanges];
  unsigned long long empty[kWorkers][kStages];  // tcgen05.commit: the operand stage has been read
  unsigned long long acc_full[kWorkers];        // tcgen05.commit: the element's MMAs are done
  unsigned long long acc_empty[kWorkers];       // 4 arrivals: every epilogue quarter has read it
  unsigned long long fin[kWorkers];             // tcgen05.commit at worker exit
  unsigned long long qfull[kQ];                 // queue entry written
  int qe[kQ];
  int qb[kQ];
  int q_head;
  int progress[kWorkers];
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

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
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

// As mbar_try, but a thread whose phase is not complete sleeps in hardware until it
// completes or about kSuspendNs have passed, instead of spinning on the issue slots.
constexpr uint32_t kSuspendNs = 200000;
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

// Waits for the phase of the given parity. Returns false once the block has failed,
// or after kWaitNs without completion.
__device__ bool mbar_wait(unsigned long long* bar, uint32_t parity, const int* failed) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  for (;;) {
    if (mbar_try_sleep(bar, parity)) return true;
    if (vload(failed) || gtime() - t0 > kWaitNs) return false;
  }
}

// As mbar_wait, for waits that may legitimately last as long as a worker needs to
// get through a crowded neighbourhood: fails only after kWaitNs in which no worker
// reported progress.
__device__ bool mbar_wait_progress(TcSmem& S, unsigned long long* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  unsigned long long t0 = gtime();
  int last_sum = -1;
  for (;;) {
    if (mbar_try_sleep(bar, parity)) return true;
    if (vload(&S.failed)) return false;
    const unsigned long long now = gtime();
    if (now - t0 > kWaitNs) {
      int sum = 0;
      for (int k = 0; k < kWorkers; ++k) sum += vload(&S.progress[k]);
      if (sum == last_sum) return false;
      last_sum = sum;
      t0 = now;
    }
  }
}

__device__ __forceinline__ void fail_now(TcSmem& S, unsigned long long* counters) {
  vstore(&S.failed, 1);
  atomicMax(counters, (unsigned long long)PC_ETIMEOUT);
}

// Queue push by a worker's lane 0: (element, worker) or the exit sentinel e = -1.
__device__ __forceinline__ void queue_push(TcSmem& S, int e, int k) {
  const int t = atomicAdd(&S.q_head, 1);
  S.qe[t % kQ] = e;
  S.qb[t % kQ] = k;
  mbar_arrive(&S.qfull[t % kQ]);  // release: the entry is visible to the waiter
}

// Worker warp k: takes the next element from the ticket counter until none is left.
// Per element: the (2 rho + 1)^3 neighbour cell ranges and their prefix sum, then an
// ordered warp-level compaction of the particles whose support reaches the element
// (per-axis reach bits) into the ring; per 32 kept particles, lane p computes the
// factors of particle p (kx scaled by 2^4, kz by 2^8) and writes its A rows
// ky_j kz_k and B rows q_c kx_i, hi and lo, into the stage, and lane 0 issues the
// MMAs. Accumulation order inside an element is the kept order, so the deposit is
// deterministic.
template <int kBf16, int N1>
__device__ void tc_worker(TcSmem& S, const TcDepositArgs& A, uint32_t tmem, uint32_t idesc, int k, int lane) {
  constexpr int NODES = N1 * N1 * N1;
  constexpr unsigned nmask = (1u << N1) - 1u;
  const int ne = A.ne, rho = A.rho, span = 2 * rho + 1, nrange = span * span * span;
  const int64_t nel = (int64_t)ne * ne * ne;
  const uint32_t acc = tmem + 64u * (uint32_t)k;
  float sv[N1];
#pragma unroll
  for (int i = 0; i < N1; ++i) sv[i] = A.s[i];
  const float c2l = A.c2l;
  // this lane's 16-byte pieces in the stages: particle octet (lane / 8), row lane % 8
  const int pa = (lane >> 3) * (kAStage / 4) + (lane & 7) * 16;
  const int pb = (lane >> 3) * (kBStage / 4) + (lane & 7) * 16;
  int chunk = 0, prog = 0, used = 0;
  bool ok = true;
  // elements in ticket order from a device counter: the elements in flight stay a
  // contiguous stretch of the mesh, so their neighbourhoods share the L2
  auto grab = [&]() -> int64_t {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(&A.counters[CNT_ELEM], 1ull);
    return (int64_t)__shfl_sync(kFull, t, 0);
  };
  for (int64_t e = grab(); ok && e < nel; e = grab()) {
    if (__any_sync(kFull, vload(&S.failed))) break;
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
        S.rbeg[k][r] = b0;
        // window element offsets as bit positions of the reach word
        S.rmeta[k][r] = (rho - dx) | ((8 + rho - dy) << 8) | ((16 + rho - dz) << 16);
      }
      int x = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
      }
      if (r < nrange) S.pre[k][r + 1] = total + x;
      total += __shfl_sync(kFull, x, 31);
    }
    if (lane == 0) S.pre[k][0] = 0;
    __syncwarp();
    int nmma = 0, scan = 0, head = 0, tail = 0;  // kept-particle ring: [head, tail)
    int rlo = 0;                                 // range holding the batch's first candidate
    // candidate batch [scan, scan + 32), loaded one batch ahead
    float4 c0r, c1r, c2r, c3r;
    int cm = 0;
    bool cvalid = false;
    auto load_batch = [&](int base) {
      const int idx = base + lane;
      cvalid = idx < total;
      int r = rlo;
      if (cvalid) {
        while (S.pre[k][r + 1] <= idx) ++r;
        cm = S.rmeta[k][r];
        const int64_t j = (int64_t)S.rbeg[k][r] + (idx - S.pre[k][r]);
        c0r = A.rec[4 * j];
        c1r = A.rec[4 * j + 1];
        c2r = A.rec[4 * j + 2];
        c3r = A.rec[4 * j + 3];
      }
      rlo = __shfl_sync(kFull, r, 0);  // the next batch starts at or after this lane's range
    };
    if (total > 0) load_batch(0);
    for (;;) {
      // refill until the ring holds more than a chunk or the neighbourhood is
      // exhausted, so that "last chunk of the element" is known exactly
      while (scan < total && tail - head <= kChunk) {
        bool keep = false;
        if (cvalid) {
          const unsigned R = __float_as_uint(c3r.y);
          keep = ((R >> (cm & 31)) & (R >> ((cm >> 8) & 31)) & (R >> ((cm >> 16) & 31)) & 1u) != 0u;
        }
        const unsigned bal = __ballot_sync(kFull, keep);
        if (keep) {
          const int pos = (tail + __popc(bal & ((1u << lane) - 1u))) & (kList - 1);
          S.lrec[k][0][pos] = c0r;
          S.lrec[k][1][pos] = c1r;
          S.lrec[k][2][pos] = c2r;
          S.lrec[k][3][pos] = c3r;
          S.lmeta[k][pos] = cm;
        }
        tail += __popc(bal);
        scan += 32;
        if (scan < total) load_batch(scan);
        if (lane == 0) vstore(&S.progress[k], ++prog);
      }
      __syncwarp();
      const int avail = tail - head;
      if (avail == 0) break;
      const int take = avail < kChunk ? avail : kChunk;
      const bool last = avail <= kChunk;  // the refill stopped short only because the scan is done
      const int st = chunk % kStages;
      // the MMAs of chunk - kStages have read this stage
      const bool free_stage =
          chunk < kStages || mbar_wait(&S.empty[k][st], (uint32_t)((chunk / kStages - 1) & 1), &S.failed);
      if (!__all_sync(kFull, free_stage)) {
        if (lane == 0) fail_now(S, A.counters + CNT_STATUS);
        ok = false;
        break;
      }
      // particle `lane` of the chunk (lanes beyond `take` build zero rows)
      const bool live = lane < take;
      const int pos = (head + lane) & (kList - 1);
      const int meta = S.lmeta[k][pos];
      const float4 r0 = S.lrec[k][0][pos], r1 = S.lrec[k][1][pos], r2 = S.lrec[k][2][pos], r3 = S.lrec[k][3][pos];
      // the 1-D factors of axis a over the element's n1 nodes: kx scaled by 2^4, kz by 2^8
      auto axis = [&](int a, float* f) {
        const float t = a == 0 ? r0.x : (a == 1 ? r0.y : r0.z);
        const float iz = a == 0 ? r0.w * 16.0f : (a == 1 ? r1.x : r1.y * 256.0f);
        const unsigned mk = __float_as_uint(a == 0 ? r2.z : (a == 1 ? r2.w : r3.x));
        const int wo = ((meta >> (8 * a)) & 31) - 8 * a;
        const int sh = wo * N1;
        const unsigned bits = live ? (sh < 32 ? (mk >> sh) : 0u) & nmask : 0u;
        const float base = (float)(wo - rho) - t;
        // pairs of nodes on the packed FP32x2 instructions (the same IEEE operations)
#pragma unroll
        for (int i = 0; i + 1 < N1; i += 2) {
          const float2 d = __fadd2_rn(make_float2(base, base), make_float2(sv[i], sv[i + 1]));
          const float2 x = __fmul2_rn(__fmul2_rn(d, d), make_float2(-c2l, -c2l));
          const float2 g = __fmul2_rn(make_float2(ex2(x.x), ex2(x.y)), make_float2(iz, iz));
          f[i] = ((bits >> i) & 1u) ? g.x : 0.0f;
          f[i + 1] = ((bits >> (i + 1)) & 1u) ? g.y : 0.0f;
        }
        if (N1 & 1) {
          const float d = base + sv[N1 - 1];
          const float g = ex2((d * d) * -c2l) * iz;
          f[N1 - 1] = ((bits >> (N1 - 1)) & 1u) ? g : 0.0f;
        }
      };
      float fy[N1], fz[N1];
      axis(1, fy);
      axis(2, fz);
      // A rows jk = j + N1 k in groups of 8: YZ_hi of group g in row group
      // 4 (g / 2) + g % 2, YZ_lo in row group 4 (g / 2) + 2 + g % 2
      uint8_t* ta = S.a[k][st] + pa;
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        if (8 * g < N1 * N1) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int jk0 = 8 * g + 2 * u, jk1 = jk0 + 1;
            float2 v;
            if (jk1 < N1 * N1 && jk0 / N1 == jk1 / N1)
              v = __fmul2_rn(make_float2(fy[jk0 % N1], fy[jk1 % N1]), make_float2(fz[jk0 / N1], fz[jk0 / N1]));
            else
              v = make_float2(jk0 < N1 * N1 ? fy[jk0 % N1] * fz[jk0 / N1] : 0.0f,
                              jk1 < N1 * N1 ? fy[jk1 % N1] * fz[jk1 / N1] : 0.0f);
            split2<kBf16>(v.x, v.y, &hi[u], &lo[u]);
          }
          const int mg = 4 * (g >> 1) + (g & 1);
          *reinterpret_cast<uint4*>(ta + 128 * mg) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(ta + 128 * (mg + 2)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
      // B rows ci = c N1 + i: A_hi in row groups 0..3, A_lo in 4..7
      float fx[N1];
      axis(0, fx);
      const float qv[4] = {live ? r1.z : 0.0f, live ? r1.w : 0.0f, live ? r2.x : 0.0f, live ? r2.y : 0.0f};
      uint8_t* tb = S.b[k][st] + pb;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        if (8 * g < 4 * N1) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c0 = 8 * g + 2 * u, c1 = c0 + 1;
            const float v0 = c0 < 4 * N1 ? qv[c0 / N1] * fx[c0 % N1] : 0.0f;
            const float v1 = c1 < 4 * N1 ? qv[c1 / N1] * fx[c1 % N1] : 0.0f;
            split2<kBf16>(v0, v1, &hi[u], &lo[u]);
          }
          *reinterpret_cast<uint4*>(tb + 128 * g) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(tb + 128 * (4 + g)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      const bool first = nmma == 0;
      if (lane == 0) {
        bool go = true;
        if (first && used > 0)  // the epilogue has read this accumulator's previous element
          go = mbar_wait(&S.acc_empty[k], (uint32_t)((used - 1) & 1), &S.failed);
        if (go) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t da = make_desc(smem_u32(S.a[k][st]), kAStage / 4, 128);
          const uint64_t db = make_desc(smem_u32(S.b[k][st]), kBStage / 4, 128);
          mma_issue(acc, da, db, idesc, first ? 0u : 1u);
          // particles 16..31: two particle octets further
          if (take > 16) mma_issue(acc, da + (uint64_t)(kAStage / 32), db + (uint64_t)(kBStage / 32), idesc, 1u);
          mma_commit(&S.empty[k][st]);
          if (last) {
            mma_commit(&S.acc_full[k]);
            queue_push(S, (int)e, k);
          }
        } else {
          fail_now(S, A.counters + CNT_STATUS);
        }
      }
      if (first) ++used;
      head += take;
      ++nmma;
      ++chunk;
      if (__shfl_sync(kFull, vload(&S.failed), 0)) {
        ok = false;
        break;
      }
      if (last) break;
    }
    if (ok && nmma == 0) {
      float* out = A.field + e * 4 * NODES;
      for (int t = lane; t < 4 * NODES; t += 32) out[t] = 0.0f;
    }
  }
  __syncwarp();
  if (lane == 0) {
    // every MMA this thread issued has completed once this commit arrives
    mma_commit(&S.fin[k]);
    int never = 0;
    (void)mbar_wait(&S.fin[k], 0, &never);
    queue_push(S, -1, k);
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float r[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) r[c] = __uint_as_float(u[c]);
}

// Epilogue warp for TMEM lane quarter q: drains the finished-element queue in
// order until every worker has sent its exit sentinel. Its lanes 0..15 hold the
// YZ_hi rows of jk = 16 q + lane and lanes 16..31 the YZ_lo rows of the same jk;
// accumulator columns 0..31 the products with A_hi, 32..63 those with A_lo. The four
// quarters work independently; each arrives on the accumulator's empty barrier as
// soon as it has read it.
template <int N1>
__device__ void tc_epilogue(TcSmem& S, const TcDepositArgs& A, uint32_t tmem, int q, int lane) {
  constexpr int NODES = N1 * N1 * N1;
  unsigned seen = 0u;  // bit k: parity of the next acc_full phase of worker k
  int exited = 0;
  for (int t = 0; exited < kWorkers; ++t) {
    if (!mbar_wait_progress(S, &S.qfull[t % kQ], (uint32_t)((t / kQ) & 1))) {
      if (lane == 0 && q == 0 && !vload(&S.failed)) fail_now(S, A.counters + CNT_STATUS);
      return;
    }
    const int e = vload(&S.qe[t % kQ]), k = vload(&S.qb[t % kQ]);
    if (e < 0) {
      ++exited;
      continue;
    }
    if (!mbar_wait(&S.acc_full[k], (seen >> k) & 1u, &S.failed)) {
      if (lane == 0) fail_now(S, A.counters + CNT_STATUS);
      return;
    }
    seen ^= 1u << k;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tq = tmem + 64u * k + ((uint32_t)(32 * q) << 16);
    float v[32];
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      float r0[16], r1[16];
      tmem_ld16(tq + 16u * hf, r0);
      tmem_ld16(tq + 32u + 16u * hf, r1);
#pragma unroll
      for (int cc = 0; cc < 16; ++cc) v[16 * hf + cc] = r0[cc] + r1[cc];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.acc_empty[k]);
    // hi rows plus lo rows
#pragma unroll
    for (int ci = 0; ci < 32; ++ci) v[ci] = v[ci] + __shfl_down_sync(kFull, v[ci], 16);
    const int jk = 16 * q + lane;
    if (lane < 16 && jk < N1 * N1) {
      float* out = A.field + (int64_t)e * 4 * NODES + jk * N1;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if constexpr (N1 % 4 == 0) {
#pragma unroll
          for (int i = 0; i < N1; i += 4)
            *reinterpret_cast<float4*>(out + c * NODES + i) =
                make_float4(v[c * N1 + i] * A.scale_out, v[c * N1 + i + 1] * A.scale_out,
                            v[c * N1 + i + 2] * A.scale_out, v[c * N1 + i + 3] * A.scale_out);
        } else {
#pragma unroll
          for (int i = 0; i < N1; ++i) out[c * NODES + i] = v[c * N1 + i] * A.scale_out;
        }
      }
    }
  }
}

template <int kBf16, int N1>
__global__ void __launch_bounds__(kThreads, 1) k_tc_deposit(TcDepositArgs A) {
  extern __shared__ uint8_t smraw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // rows no lane writes (n1 < 8) stay zero
  for (int i = tid; i < kWorkers * kStages * kAStage / 16; i += kThreads)
    reinterpret_cast<uint4*>(&S.a[0][0][0])[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < kWorkers * kStages * kBStage / 16; i += kThreads)
    reinterpret_cast<uint4*>(&S.b[0][0][0])[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int k = 0; k < kWorkers; ++k) {
      for (int s = 0; s < kStages; ++s)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.empty[k][s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.acc_full[k])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&S.acc_empty[k])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.fin[k])));
      S.progress[k] = 0;
    }
    for (int t = 0; t < kQ; ++t) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.qfull[t])));
    S.q_head = 0;
    S.failed = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem_base;
  // D FP32, A and B FP16 or BF16, both MN-major (transposed), N = 64, M = 128
  const uint32_t fmt = kBf16 ? 1u : 0u;
  const uint32_t idesc =
      (1u << 4) | (fmt << 7) | (fmt << 10) | (1u << 15) | (1u << 16) | (8u << 17) | (8u << 24);
  if (warp < kWorkers)
    tc_worker<kBf16, N1>(S, A, tmem, idesc, warp, lane);
  else
    tc_epilogue<N1>(S, A, tmem, warp % 4, lane);  // a warp reaches the TMEM lane quarter warp % 4
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

template <int kBf16, int N1>
cudaError_t tc_launch(const TcDepositArgs& A, int grid, size_t smem, cudaStream_t st) {
  PC_CUDA_TRY(cudaFuncSetAttribute(k_tc_deposit<kBf16, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_tc_deposit<kBf16, N1><<<(unsigned)grid, kThreads, smem, st>>>(A);
  return cudaGetLastError();
}

template <int kBf16>
cudaError_t tc_launch_n1(const TcDepositArgs& A, int grid, size_t smem, cudaStream_t st) {
  switch (A.n1) {
    case 1: return tc_launch<kBf16, 1>(A, grid, smem, st);
    case 2: return tc_launch<kBf16, 2>(A, grid, smem, st);
    case 3: return tc_launch<kBf16, 3>(A, grid, smem, st);
    case 4: return tc_launch<kBf16, 4>(A, grid, smem, st);
    case 5: return tc_launch<kBf16, 5>(A, grid, smem, st);
    case 6: return tc_launch<kBf16, 6>(A, grid, smem, st);
    case 7: return tc_launch<kBf16, 7>(A, grid, smem, st);
    case 8: return tc_launch<kBf16, 8>(A, grid, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t pc_tc_deposit_launch(const TcDepositArgs& A, cudaStream_t st, int* nblocks) {
  const size_t smem = sizeof(TcSmem) + 1024;
  const int64_t nel = (int64_t)A.ne * A.ne * A.ne;
  int dev = 0, sms = 0;
  PC_CUDA_TRY(cudaGetDevice(&dev));
  PC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // one persistent CTA per SM: it holds all 512 tensor-memory columns
  int64_t grid = (nel + kWorkers - 1) / kWorkers;
  if (grid > sms) grid = sms;
  if (grid < 1) grid = 1;
  *nblocks = (int)grid;
  return A.tc_type == PC_TC_BF16 ? tc_launch_n1<1>(A, (int)grid, smem, st) : tc_launch_n1<0>(A, (int)grid, smem, st);
}
