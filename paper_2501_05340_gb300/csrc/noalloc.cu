// pc_project_noalloc: the projection for callers that may not allocate device
// memory, e.g. a plugin inside a host solver whose memory manager owns the whole
// GPU and forbids allocations by anyone else, or a time-critical loop where an
// allocation's latency or failure is not acceptable. It runs the same kernels as
// pc_project, with all scratch taken from one fixed device array compiled into
// the library instead of from a context.
#include <math.h>
#include <string.h>

#include <cuda.h>

#include <mutex>

#include "pc_internal.cuh"

namespace {

// Scratch of pc_project_noalloc. Every GPU that loads the library holds it until
// the process exits.
constexpr size_t kNoallocBytes = (size_t)PC_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch per device. In host code the array's name
// is only a host-side stand-in, so the address is looked up once per device and
// context: a cudaDeviceReset destroys the context that held the array, and the
// next call sees a context with another id and looks the address up again.
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];
std::mutex g_scratch_mu;

// Driver entry points for the current context's unique id (no link to libcuda:
// the runtime hands out the driver's functions).
typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);
ctx_get_current_fn g_ctx_current;
ctx_get_id_fn g_ctx_id;

// Unique id of the calling thread's current context, 0 if there is none or the
// driver cannot tell.
unsigned long long current_context_id() {
  if (!g_ctx_current || !g_ctx_id) {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess)
      return 0;
    g_ctx_current = (ctx_get_current_fn)a;
    g_ctx_id = (ctx_get_id_fn)b;
  }
  CUcontext cu = nullptr;
  unsigned long long id = 0;
  if (g_ctx_current(&cu) != CUDA_SUCCESS || !cu || g_ctx_id(cu, &id) != CUDA_SUCCESS) return 0;
  return id;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

void put_msg(char* msg, int64_t len, const char* text) {
  if (msg && len > 0) {
    strncpy(msg, text, (size_t)len - 1);
    msg[len - 1] = '\0';
  }
}

}  // namespace

extern "C" pc_status pc_project_noalloc(const pc_config* cfg, const pc_particles* p, double* field, char* msg,
                                        int64_t msg_len) {
  put_msg(msg, msg_len, "no error");
  if (!cfg || !p || !field || p->n < 0 || (p->n > 0 && (!p->x || !p->q || !p->id))) {
    put_msg(msg, msg_len, "pc_project_noalloc: bad arguments");
    return PC_EINVAL;
  }
  // particle indices and bin slots are int32 on the device
  if (p->n >= ((int64_t)1 << 31)) {
    put_msg(msg, msg_len, "pc_project_noalloc: more than 2^31 - 1 particles");
    return PC_EINVAL;
  }
  const pc_config& c = *cfg;
  if (c.ne < 3 || c.ne > 1024 || c.degree < 0 || c.degree > 15 || !(c.sigma > 0.0) || !(c.cutoff_sigmas > 0.0) ||
      c.cutoff_kind != 0) {
    put_msg(msg, msg_len, "pc_project_noalloc: bad configuration");
    return PC_EINVAL;
  }
  const double rc = c.cutoff_sigmas * c.sigma;
  const int rho = (int)ceil(rc * c.ne * (1.0 + 1e-12));
  if (rho < 1 || rho > 2 || 2 * rho + 1 > c.ne || !(rc < 0.5) || (2 * rho + 1) * (c.degree + 1) > 64) {
    put_msg(msg, msg_len, "pc_project_noalloc: cutoff out of range for the mesh");
    return PC_EINVAL;
  }
  const int64_t n = p->n;
  const int n1 = c.degree + 1;
  const int win = (2 * rho + 1) * n1;
  const int64_t nel = (int64_t)c.ne * c.ne * c.ne;

  // carve the fixed array: counters, bin counts and starts, scan block sums,
  // key/slot/perm, factors, sources
  size_t off = 0;
  const size_t o_cnt_ctr = off;
  off = align256(off + sizeof(unsigned long long) * CNT_N);
  const size_t o_cnt = off;
  off = align256(off + sizeof(int32_t) * (size_t)(nel + 1));
  const size_t o_start = off;
  off = align256(off + sizeof(int32_t) * (size_t)(nel + 1));
  const size_t o_bs = off;
  off = align256(off + sizeof(int32_t) * (size_t)((nel + 1) / PC_SCAN_TILE + 2));
  const size_t o_key = off;
  off = align256(off + sizeof(int32_t) * (size_t)n);
  const size_t o_slot = off;
  off = align256(off + sizeof(int32_t) * (size_t)n);
  const size_t o_perm = off;
  off = align256(off + sizeof(int32_t) * (size_t)n);
  const int rs = (3 * win + 4 + 1) & ~1;
  const size_t o_fac = off;
  off = align256(off + sizeof(float2) * (size_t)rs * (size_t)n);
  const size_t o_sq = off;
  off = align256(off + sizeof(float2) * (size_t)4 * (size_t)n);
  const size_t o_reach = off;
  off = align256(off + sizeof(int32_t) * (size_t)n);
  const size_t o_fxmax = off;
  off = align256(off + sizeof(unsigned) * 8);
  if (off > kNoallocBytes) {
    char text[200];
    snprintf(text, sizeof(text),
             "pc_project_noalloc: needs %zu bytes of scratch, the fixed array holds %zu (fewer particles or "
             "a coarser mesh, or use pc_init + pc_project)",
             off, kNoallocBytes);
    put_msg(msg, msg_len, text);
    return PC_ECAPACITY;
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    put_msg(msg, msg_len, "pc_project_noalloc: no usable CUDA device");
    return PC_ECUDA;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long cid = current_context_id();
    if (!g_scratch_addr[dev] || cid == 0 || cid != g_scratch_ctx[dev]) {
      void* a = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
      if (e != cudaSuccess || !a) {
        put_msg(msg, msg_len, "pc_project_noalloc: cudaGetSymbolAddress failed");
        return PC_ECUDA;
      }
      g_scratch_addr[dev] = a;
      // the lookup makes the device's primary context current if none was
      g_scratch_ctx[dev] = current_context_id();
    }
    base = (unsigned char*)g_scratch_addr[dev];
  }

  // a context on the stack that points into the fixed array (timing off)
  pc_ctx ctx;
  memset(&ctx, 0, sizeof(ctx));
  ctx.cfg = c;
  ctx.stream = (cudaStream_t)c.stream;
  ctx.device = dev;
  ctx.n1 = n1;
  ctx.rho = rho;
  ctx.win = win;
  ctx.h = 1.0 / c.ne;
  pc_gauss_rule(n1, ctx.eta, ctx.w);
  pc_build_exp_table(&ctx.exp_tab);
  ctx.counters = (unsigned long long*)(base + o_cnt_ctr);
  ctx.cnt = (int32_t*)(base + o_cnt);
  ctx.start = (int32_t*)(base + o_start);
  ctx.blocksums = (int32_t*)(base + o_bs);
  ctx.key = (int32_t*)(base + o_key);
  ctx.slot = (int32_t*)(base + o_slot);
  ctx.perm = (int32_t*)(base + o_perm);
  ctx.rs = rs;
  ctx.fac = (float2*)(base + o_fac);
  ctx.sq = (float2*)(base + o_sq);
  ctx.reach = (int32_t*)(base + o_reach);
  ctx.fxmax = (unsigned*)(base + o_fxmax);
  // the array keeps the previous call's contents: clear the status counters
  if (cudaMemsetAsync(ctx.counters, 0, sizeof(unsigned long long) * CNT_N, ctx.stream) != cudaSuccess) {
    put_msg(msg, msg_len, "pc_project_noalloc: cudaMemsetAsync failed");
    return PC_ECUDA;
  }
  const pc_status s = pc_project_impl(&ctx, p, field);
  if (s != PC_OK) put_msg(msg, msg_len, ctx.err);
  return s;
}
