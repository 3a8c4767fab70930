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

constexpr int kThreads = 128;
constexpr int kStages = 4;
constexpr int kChunk = 16;
constexpr int kListMax = 2048;
constexpr uint32_t kTmemCols = 64;
constexpr long kSpinLimit = 1L << 26;

struct __align__(1024) TcSmem {
  uint8_t a[kStages][4096];
  uint8_t b[kStages][2048];
  float pf[kStages][kChunk][28];  // kx[8] ky[8] kz[8] q[4] per staged particle
  float comb[64][33];
  int list[kListMax];
  int lmeta[kListMax];
  int pre[128];
  int rbeg[128];
  int wcount[4];
  unsigned long long mbar_stage[kStages];
  unsigned long long mbar_done;
  uint32_t tmem_base;
  int nlist;
  int failed;
};

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

template <int kBf16>
__global__ void __launch_bounds__(kThreads) k_tc_deposit(TcDepositArgs A) {
  extern __shared__ uint8_t smraw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n1 = A.n1, ne = A.ne, rho = A.rho, span = 2 * rho + 1, nrange = span * span * span;
  const int nodes = n1 * n1 * n1;
  const int64_t nel = (int64_t)ne * ne * ne;

  for (int i = tid; i < kStages * 4096 / 16; i += kThreads) reinterpret_cast<uint4*>(&S.a[0][0])[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < kStages * 2048 / 16; i += kThreads) reinterpret_cast<uint4*>(&S.b[0][0])[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar_stage[s])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar_done)));
    S.failed = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem_base;
  // kind::f16, D = F32, A/B = F16 (0) or BF16 (1), both K-major, N = 64, M = 128
  const uint32_t fmt = kBf16 ? 1u : 0u;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (8u << 17) | (8u << 24);
  long chunk_counter = 0;
  uint32_t done_count = 0;

  for (int64_t e = blockIdx.x; e < nel; e += gridDim.x) {
    if (S.failed) break;
    const int ex = (int)(e % ne), ey = (int)((e / ne) % ne), ez = (int)(e / ((int64_t)ne * ne));
    if (tid == 0) {
      int s = 0;
      for (int r = 0; r < nrange; ++r) {
        const int dx = r % span - rho, dy = (r / span) % span - rho, dz = r / (span * span) - rho;
        const int nb = (wrapi(ez + dz, ne) * ne + wrapi(ey + dy, ne)) * ne + wrapi(ex + dx, ne);
        const int b0 = A.start[nb], b1 = A.start[nb + 1];
        S.pre[r] = s;
        S.rbeg[r] = b0;
        s += b1 - b0;
      }
      S.pre[nrange] = s;
    }
    __syncthreads();
    const int total = S.pre[nrange];
    int nmma = 0;
    int scan = 0;
    while (scan < total && !S.failed) {
      // ---- ordered compaction of the particles whose support reaches this element
      if (tid == 0) S.nlist = 0;
      __syncthreads();
      while (scan < total) {
        const int idx = scan + tid;
        bool keep = false;
        int j = 0, meta = 0;
        if (idx < total) {
          int r = 0;
          while (S.pre[r + 1] <= idx) ++r;
          j = S.rbeg[r] + (idx - S.pre[r]);
          const int d3[3] = {r % span - rho, (r / span) % span - rho, r / (span * span) - rho};
          const float4 r2 = A.rec[4 * (int64_t)j + 2];
          const float4 r3 = A.rec[4 * (int64_t)j + 3];
          const unsigned mk[3] = {__float_as_uint(r2.z), __float_as_uint(r2.w), __float_as_uint(r3.x)};
          keep = true;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int wo = rho - d3[a];  // this element's slot in the particle's window
            keep = keep && ((mk[a] >> (wo * n1)) & ((1u << n1) - 1u)) != 0u;
            meta |= wo << (4 * a);
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) S.wcount[warp] = __popc(bal);
        __syncthreads();
        int base = S.nlist;
        for (int w = 0; w < warp; ++w) base += S.wcount[w];
        const int added = S.wcount[0] + S.wcount[1] + S.wcount[2] + S.wcount[3];
        if (keep) {
          const int pos = base + __popc(bal & ((1u << lane) - 1u));
          S.list[pos] = j;
          S.lmeta[pos] = meta;
        }
        __syncthreads();
        if (tid == 0) S.nlist += added;
        scan += kThreads;
        __syncthreads();
        if (S.nlist + kThreads > kListMax) break;
      }
      const int nl = S.nlist;
      // ---- chunks of 16 kept particles: stage factors, build operands, one MMA
      for (int c0 = 0; c0 < nl; c0 += kChunk) {
        const int s = (int)(chunk_counter % kStages);
        if (chunk_counter >= kStages) {
          const uint32_t par = (uint32_t)((chunk_counter / kStages - 1) & 1);
          if (!mbar_wait(&S.mbar_stage[s], par)) {
            atomicMax(&A.counters[CNT_STATUS], (unsigned long long)PC_ETIMEOUT);
            S.failed = 1;
          }
        }
        __syncthreads();
        if (S.failed) break;
        {
          const int p = tid >> 3, i = tid & 7;
          float f3[3] = {0.0f, 0.0f, 0.0f}, qv = 0.0f;
          if (c0 + p < nl && i < n1) {
            const int64_t j = S.list[c0 + p];
            const int meta = S.lmeta[c0 + p];
            const float4 r0 = A.rec[4 * j], r1 = A.rec[4 * j + 1], r2 = A.rec[4 * j + 2], r3 = A.rec[4 * j + 3];
            const float t3[3] = {r0.x, r0.y, r0.z}, iz[3] = {r0.w, r1.x, r1.y};
            const unsigned mk[3] = {__float_as_uint(r2.z), __float_as_uint(r2.w), __float_as_uint(r3.x)};
            const float q4[4] = {r1.z, r1.w, r2.x, r2.y};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const int wo = (meta >> (4 * a)) & 15;
              const int w = wo * n1 + i;
              if ((mk[a] >> w) & 1u) {
                const float d = (float)(wo - rho) + A.s[i] - t3[a];
                f3[a] = exp2f(-(d * d) * A.c2l) * iz[a];
              }
            }
            if (i < 4) qv = q4[i];
          }
          float* pf = S.pf[s][p];
          pf[i] = f3[0];
          pf[8 + i] = f3[1];
          pf[16 + i] = f3[2];
          if (i < 4) pf[24 + i] = qv;
        }
        __syncthreads();
        if (tid < 64) {
          const int jk = tid;
          if (jk < n1 * n1) {
            const int jj = jk % n1, kk = jk / n1;
            float v[16];
#pragma unroll
            for (int p = 0; p < kChunk; ++p) v[p] = S.pf[s][p][8 + jj] * S.pf[s][p][16 + kk] * 256.0f;
            store_row<kBf16>(S.a[s], jk, 64, v);
          }
        } else if (tid < 96) {
          const int ci = tid - 64;
          if (ci < 4 * n1) {
            const int c = ci / n1, i = ci % n1;
            float v[16];
#pragma unroll
            for (int p = 0; p < kChunk; ++p) v[p] = S.pf[s][p][24 + c] * S.pf[s][p][i] * 16.0f;
            store_row<kBf16>(S.b[s], ci, 32, v);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          mma_issue(tmem, make_desc(smem_u32(S.a[s]), 128, 256), make_desc(smem_u32(S.b[s]), 128, 256), idesc,
                    nmma > 0 ? 1u : 0u);
          mma_commit(&S.mbar_stage[s]);
        }
        ++nmma;
        ++chunk_counter;
      }
    }
    if (S.failed) break;
    float* out = A.field + e * 4 * nodes;
    if (nmma == 0) {
      for (int a = tid; a < 4 * nodes; a += kThreads) out[a] = 0.0f;
      __syncthreads();
      continue;
    }
    // ---- epilogue: wait for the element's MMAs, add the four quadrants
    if (tid == 0) mma_commit(&S.mbar_done);
    if (!mbar_wait(&S.mbar_done, done_count & 1)) {
      atomicMax(&A.counters[CNT_STATUS], (unsigned long long)PC_ETIMEOUT);
      S.failed = 1;
    }
    ++done_count;
    __syncthreads();
    if (S.failed) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float r[64];
    tmem_ld64(tmem + ((uint32_t)(32 * warp) << 16), r);
    const int jk = 32 * (warp & 1) + lane;
    if (warp >= 2) {
#pragma unroll
      for (int ci = 0; ci < 32; ++ci) S.comb[jk][ci] = r[ci] + r[32 + ci];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp < 2 && jk < n1 * n1) {
      for (int ci = 0; ci < 4 * n1; ++ci) {
        const int c = ci / n1, i = ci % n1;
        out[c * nodes + jk * n1 + i] = ((r[ci] + r[32 + ci]) + S.comb[jk][ci]) * A.scale_out;
      }
    }
    __syncthreads();
  }
  // ---- teardown: no MMA may be in flight when the tensor memory is freed
  if (S.failed) {
    if (tid == 0) mma_commit(&S.mbar_done);
    (void)mbar_wait(&S.mbar_done, done_count & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

cudaError_t pc_tc_deposit_launch(const TcDepositArgs& A, cudaStream_t st, int* nblocks) {
  const size_t smem = sizeof(TcSmem) + 1024;
  const int64_t nel = (int64_t)A.ne * A.ne * A.ne;
  int dev = 0, sms = 0, per = 0;
  PC_CUDA_TRY(cudaGetDevice(&dev));
  PC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (A.tc_type == PC_TC_BF16) {
    PC_CUDA_TRY(cudaFuncSetAttribute(k_tc_deposit<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tc_deposit<1>, kThreads, smem));
  } else {
    PC_CUDA_TRY(cudaFuncSetAttribute(k_tc_deposit<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tc_deposit<0>, kThreads, smem));
  }
  if (per < 1) per = 1;
  if (per > 4) per = 4;  // 4 x 64 tensor-memory columns per SM at most
  int64_t grid = (int64_t)sms * per;
  if (grid > nel) grid = nel;
  if (grid < 1) grid = 1;
  *nblocks = (int)grid;
  if (A.tc_type == PC_TC_BF16)
    k_tc_deposit<1><<<(unsigned)grid, kThreads, smem, st>>>(A);
  else
    k_tc_deposit<0><<<(unsigned)grid, kThreads, smem, st>>>(A);
  return cudaGetLastError();
}
