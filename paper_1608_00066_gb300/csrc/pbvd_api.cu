// Host side of the C ABI declared in include/pbvd.h: argument checks, kernel
// selection, workspace management and launches.  No decoding arithmetic runs
// on the host.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "pbvd.h"
#include "pbvd_internal.h"

using namespace pbvd;

namespace {

std::mutex g_err_mu;
char g_last_cuda[256] = "no error";

int cuda_fail(cudaError_t e) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  std::snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PBVD_ENOMEM : PBVD_ECUDA;
}

#define PBVD_CUDA(call)                     \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

struct Registry {
  std::vector<KernelEntry> entries;
  std::vector<int> smem_set;  // max dynamic smem already granted per entry
};

Registry& registry() {
  static Registry reg;
  static std::once_flag once;
  std::call_once(once, [] {
    KernelEntry buf[64];
    int n = 0;
    n += register_k7(buf + n, 64 - n);
    n += register_k9(buf + n, 64 - n);
    n += register_small(buf + n, 64 - n);
    reg.entries.assign(buf, buf + n);
    reg.smem_set.assign(n, 48 * 1024);
  });
  return reg;
}
std::mutex g_reg_mu;

int find_entry(int K, int R, const uint32_t* gens, int T, bool punct) {
  Registry& reg = registry();
  for (size_t i = 0; i < reg.entries.size(); ++i) {
    const KernelEntry& e = reg.entries[i];
    if (e.K != K || e.R != R || e.T != T || e.punct != punct) continue;
    bool same = true;
    for (int r = 0; r < R; ++r) same = same && (e.gens[r] == gens[r]);
    if (same) return (int)i;
  }
  return -1;
}

int code_has_any_kernel(int K, int R, const uint32_t* gens, bool punct) {
  for (int T = 1; T <= 32; T *= 2)
    if (find_entry(K, R, gens, T, punct) >= 0) return 1;
  return 0;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

struct pbvd_ctx {
  int K, R, v, N;
  uint32_t gens[3];
  int P;                 // puncture period, 0 = none
  int punct_C;           // values sent per period
  uint8_t pattern[3 * 32];
  int16_t punct_off[32 * 4];
  int16_t punct_pre[33];
  int D, L;
  pbvd_config cfg;
  int device;
  int sm_count;
  int smem_optin;
  void* work;
  size_t work_bytes;
};

namespace {

// Resolved launch configuration.
struct Plan {
  int entry;
  int T;
  int cta;
  int smem_surv;
  int64_t n_blocks, n_pairs;
  int groups;            // groups per CTA
  int rec_words;         // smem-mode record words per group
  size_t smem_bytes;
  size_t surv_bytes;     // global-mode survivor bytes
};

int states_max_per_thread() { return 64; }

int plan_decode(const pbvd_ctx* c, size_t n_stages, Plan* p) {
  Registry& reg = registry();
  p->n_blocks = ceil_div((int64_t)n_stages, c->D);
  p->n_pairs = ceil_div(p->n_blocks, 2);
  int T = c->cfg.threads_per_pair;
  if (T <= 0) {
    int tmin = 1;
    while (c->N / tmin > states_max_per_thread()) tmin *= 2;
    const int64_t target = (int64_t)c->sm_count * 4 * 2 * 32;  // ~2 warps per scheduler
    int64_t want = ceil_div(target, std::max<int64_t>(p->n_pairs, 1));
    T = 1;
    while (T < want && T < 32) T *= 2;
    T = std::max(T, tmin);
    T = std::min(T, std::min(32, c->N / 2));
    while (T > tmin && find_entry(c->K, c->R, c->gens, T, c->P != 0) < 0) T /= 2;
    while (T < 32 && find_entry(c->K, c->R, c->gens, T, c->P != 0) < 0) T *= 2;
  }
  p->T = T;
  p->entry = find_entry(c->K, c->R, c->gens, T, c->P != 0);
  if (p->entry < 0) return PBVD_EUNSUPPORTED;
  const KernelEntry& e = reg.entries[p->entry];
  const int64_t jmax = (int64_t)c->D + c->L;
  p->rec_words = (int)(((jmax * e.words_per_stage) + 3) & ~3LL);
  int smem = c->cfg.survivors_in_smem;
  if (smem < 0) {
    const int64_t bytes = (int64_t)(p->rec_words + e.scratch_words) * 4;
    smem = (p->n_pairs <= c->sm_count && bytes <= 160 * 1024) ? 1 : 0;
  }
  p->smem_surv = smem;
  int cta = c->cfg.cta_threads;
  if (cta <= 0) cta = smem ? T : std::max(T, 64);
  if (cta % T != 0 || cta > 256 || cta < T) return PBVD_EINVAL;
  p->cta = cta;
  p->groups = cta / T;
  p->smem_bytes = (size_t)p->groups * e.scratch_words * 4 +
                  (smem ? (size_t)p->groups * p->rec_words * 4 : 0);
  if (p->smem_bytes > (size_t)c->smem_optin) {
    if (smem) return PBVD_EINVAL;  // too many groups per CTA for the records
    return PBVD_EINVAL;
  }
  p->surv_bytes = smem ? 0 : (size_t)jmax * (size_t)p->n_pairs * e.words_per_stage * 4;
  return PBVD_OK;
}

int ensure_work(pbvd_ctx* c, size_t bytes) {
  if (bytes <= c->work_bytes) return PBVD_OK;
  if (c->work) {
    cudaError_t e = cudaFree(c->work);
    c->work = nullptr;
    c->work_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(e);
  }
  cudaError_t e = cudaMalloc(&c->work, bytes);
  if (e != cudaSuccess) {
    c->work = nullptr;
    return cuda_fail(e);
  }
  c->work_bytes = bytes;
  return PBVD_OK;
}

int grant_smem(int entry, size_t bytes) {
  Registry& reg = registry();
  std::lock_guard<std::mutex> lk(g_reg_mu);
  if ((int)bytes <= reg.smem_set[entry]) return PBVD_OK;
  PBVD_CUDA(reg.entries[entry].set_max_smem((int)bytes));
  reg.smem_set[entry] = (int)bytes;
  return PBVD_OK;
}

}  // namespace

extern "C" {

const char* pbvd_strerror(int code) {
  switch (code) {
    case PBVD_OK: return "ok";
    case PBVD_EINVAL: return "invalid argument";
    case PBVD_ENOMEM: return "out of memory";
    case PBVD_ECUDA: return "CUDA error";
    case PBVD_EUNSUPPORTED: return "no kernel built for this code / configuration";
    case PBVD_ETIMEOUT: return "bounded device wait timed out";
    case PBVD_EBUSY: return "resource busy";
    default: return "unknown error";
  }
}

const char* pbvd_last_cuda_error(void) { return g_last_cuda; }

int pbvd_create(pbvd_ctx** out, int K, int R, const uint32_t* gens, const uint8_t* puncture, int P,
                int D, int L) {
  if (!out || !gens) return PBVD_EINVAL;
  *out = nullptr;
  if (K < 3 || K > 9 || R < 2 || R > 3) return PBVD_EINVAL;
  for (int r = 0; r < R; ++r) {
    if (gens[r] >> K) return PBVD_EINVAL;
    if (!((gens[r] >> (K - 1)) & 1u) && !(gens[r] & 1u)) return PBVD_EINVAL;
  }
  if (D <= 0 || (D % 8) != 0 || L < 0 || L > 4096 || D > (1 << 20)) return PBVD_EINVAL;
  if (puncture) {
    if (P < 1 || P > 32) return PBVD_EINVAL;
    for (int col = 0; col < P; ++col) {
      int sent = 0;
      for (int r = 0; r < R; ++r) {
        if (puncture[r * P + col] > 1) return PBVD_EINVAL;
        sent += puncture[r * P + col];
      }
      if (!sent) return PBVD_EINVAL;
    }
  }
  if (!code_has_any_kernel(K, R, gens, puncture != nullptr)) return PBVD_EUNSUPPORTED;

  pbvd_ctx* c = new (std::nothrow) pbvd_ctx();
  if (!c) return PBVD_ENOMEM;
  c->K = K;
  c->R = R;
  c->v = K - 1;
  c->N = 1 << (K - 1);
  for (int r = 0; r < 3; ++r) c->gens[r] = r < R ? gens[r] : 0u;
  c->P = puncture ? P : 0;
  std::memset(c->punct_off, 0xff, sizeof(c->punct_off));
  c->punct_C = 0;
  if (puncture) {
    int off = 0;
    for (int col = 0; col < P; ++col) {
      c->punct_pre[col] = (int16_t)off;
      for (int r = 0; r < R; ++r) {
        c->pattern[r * 32 + col] = puncture[r * P + col];
        if (puncture[r * P + col]) c->punct_off[col * 4 + r] = (int16_t)off++;
      }
    }
    c->punct_pre[P] = (int16_t)off;
    c->punct_C = off;
  }
  c->D = D;
  c->L = L;
  c->cfg.threads_per_pair = 0;
  c->cfg.cta_threads = 0;
  c->cfg.survivors_in_smem = -1;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e);
  }
  *out = c;
  return PBVD_OK;
}

void pbvd_destroy(pbvd_ctx* c) {
  if (!c) return;
  if (c->work) {
    cudaDeviceSynchronize();
    cudaFree(c->work);
  }
  delete c;
}

int pbvd_llr_count(const pbvd_ctx* c, size_t n_stages, size_t* count) {
  if (!c || !count) return PBVD_EINVAL;
  if (!c->P) {
    *count = n_stages * (size_t)c->R;
    return PBVD_OK;
  }
  size_t full = n_stages / c->P, rem = n_stages % c->P, tot = full * (size_t)c->punct_C;
  for (size_t col = 0; col < rem; ++col)
    for (int r = 0; r < c->R; ++r) tot += c->pattern[r * 32 + col];
  *count = tot;
  return PBVD_OK;
}

int pbvd_set_config(pbvd_ctx* c, const pbvd_config* cfg) {
  if (!c || !cfg) return PBVD_EINVAL;
  if (cfg->threads_per_pair != 0) {
    int T = cfg->threads_per_pair;
    if (T < 1 || T > 32 || (T & (T - 1))) return PBVD_EINVAL;
    if (find_entry(c->K, c->R, c->gens, T, c->P != 0) < 0) return PBVD_EUNSUPPORTED;
  }
  if (cfg->cta_threads != 0 && (cfg->cta_threads < 1 || cfg->cta_threads > 256)) return PBVD_EINVAL;
  if (cfg->survivors_in_smem < -1 || cfg->survivors_in_smem > 1) return PBVD_EINVAL;
  c->cfg = *cfg;
  return PBVD_OK;
}

int pbvd_get_config(const pbvd_ctx* c, size_t n_stages, pbvd_config* cfg) {
  if (!c || !cfg || n_stages == 0) return PBVD_EINVAL;
  Plan p;
  int rc = plan_decode(c, n_stages, &p);
  if (rc != PBVD_OK) return rc;
  cfg->threads_per_pair = p.T;
  cfg->cta_threads = p.cta;
  cfg->survivors_in_smem = p.smem_surv;
  return PBVD_OK;
}

int pbvd_decode(pbvd_ctx* c, const int8_t* d_llr, size_t n_stages, uint8_t* d_out, void* stream) {
  if (!c || !d_llr || !d_out || n_stages == 0) return PBVD_EINVAL;
  if (n_stages > ((size_t)1 << 40)) return PBVD_EINVAL;
  Plan p;
  int rc = plan_decode(c, n_stages, &p);
  if (rc != PBVD_OK) return rc;
  if (!p.smem_surv) {
    rc = ensure_work(c, p.surv_bytes);
    if (rc != PBVD_OK) return rc;
  }
  rc = grant_smem(p.entry, p.smem_bytes);
  if (rc != PBVD_OK) return rc;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.llr = d_llr;
  a.out = d_out;
  a.surv = static_cast<uint32_t*>(c->work);
  a.n = (int64_t)n_stages;
  a.n_blocks = p.n_blocks;
  a.n_pairs = p.n_pairs;
  a.surv_pairs = p.n_pairs;
  a.D = c->D;
  a.L = c->L;
  a.smem_surv = p.smem_surv;
  a.smem_rec_words = p.smem_surv ? p.rec_words : 0;
  a.punct_P = c->P;
  a.punct_C = c->punct_C;
  std::memcpy(a.punct_off, c->punct_off, sizeof(a.punct_off));
  std::memcpy(a.punct_pre, c->punct_pre, sizeof(a.punct_pre));
  size_t cnt = 0;
  pbvd_llr_count(c, n_stages, &cnt);
  a.llr_count = (int64_t)cnt;
  a.one = 1u;
  const int64_t grid = ceil_div(p.n_pairs, p.groups);
  if (grid > 0x7fffffff) return PBVD_EINVAL;
  const KernelEntry& e = registry().entries[p.entry];
  PBVD_CUDA(e.launch(a, (int)grid, p.cta, p.smem_bytes, static_cast<cudaStream_t>(stream)));
  return PBVD_OK;
}

int pbvd_decode_batch(const pbvd_batch_item* items, size_t n_items, void* stream) {
  if (!items && n_items) return PBVD_EINVAL;
  (void)stream;
  return PBVD_EUNSUPPORTED;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Allocation-free decode.
//
// Some callers must not allocate device memory while they decode: code that
// runs inside CUDA stream capture (an allocation there either fails or
// breaks the capture), real-time receive chains that reserve all memory at
// start-up and forbid allocation on the data path, and hosts whose device
// memory belongs to their own pool allocator.  pbvd_decode grows a per-context
// workspace with cudaMalloc on first use of a larger size; this variant keeps
// the survivor bits in one fixed array that is part of the library's device
// image instead, and calls no allocation routine.
//
// The array is file-scope device memory: every GPU that loads the library
// holds kNoAllocSurvivorBytes of it until the process exits.  Host code may
// not use the array's name as an address (on the host it is only a
// stand-in), so its device address is looked up once per device with
// cudaGetSymbolAddress while that device is current, and passed to the
// kernel.  That lookup happens on the first call on each device, so make the
// first call outside any stream capture.  All calls share the array and it
// keeps the last call's contents: nothing needs clearing (every survivor word
// the traceback reads is written earlier in the same launch), but calls whose
// work overlaps on the GPU race on it.

namespace {

constexpr size_t kNoAllocSurvivorBytes = size_t(16) << 20;  // 16 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) uint32_t g_noalloc_survivors[kNoAllocSurvivorBytes / sizeof(uint32_t)];

std::mutex g_noalloc_mu;
uint32_t* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the survivor array on the current device (looked up once).
int noalloc_survivors(int device, uint32_t** out) {
  if (device < 0 || device >= kNoAllocMaxDevices) return PBVD_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_survivors);
    if (e != cudaSuccess) return cuda_fail(e);
    g_noalloc_ptr[device] = static_cast<uint32_t*>(p);
  }
  *out = g_noalloc_ptr[device];
  return PBVD_OK;
}

}  // namespace

extern "C" {

int pbvd_decode_noalloc(pbvd_ctx* c, const int8_t* d_llr, size_t n_stages, uint8_t* d_out, void* stream) {
  if (!c || !d_llr || !d_out || n_stages == 0) return PBVD_EINVAL;
  if (n_stages > ((size_t)1 << 40)) return PBVD_EINVAL;
  int dev = -1;
  PBVD_CUDA(cudaGetDevice(&dev));
  if (dev != c->device) return PBVD_EINVAL;
  // the survivor bits always live in the fixed array here
  pbvd_ctx cc = *c;
  cc.cfg.survivors_in_smem = 0;
  Plan p;
  int rc = plan_decode(&cc, n_stages, &p);
  if (rc != PBVD_OK) return rc;
  // with an automatic thread count, fall back to fewer threads per pair
  // (smaller survivor records) until the survivor bits fit the array
  while (c->cfg.threads_per_pair == 0 && p.surv_bytes > kNoAllocSurvivorBytes && p.T > 1) {
    cc.cfg.threads_per_pair = p.T / 2;
    if (find_entry(c->K, c->R, c->gens, cc.cfg.threads_per_pair, c->P != 0) < 0) break;
    rc = plan_decode(&cc, n_stages, &p);
    if (rc != PBVD_OK) return rc;
  }
  if (p.surv_bytes > kNoAllocSurvivorBytes) return PBVD_EINVAL;
  uint32_t* surv = nullptr;
  rc = noalloc_survivors(dev, &surv);
  if (rc != PBVD_OK) return rc;
  rc = grant_smem(p.entry, p.smem_bytes);
  if (rc != PBVD_OK) return rc;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.llr = d_llr;
  a.out = d_out;
  a.surv = surv;
  a.n = (int64_t)n_stages;
  a.n_blocks = p.n_blocks;
  a.n_pairs = p.n_pairs;
  a.surv_pairs = p.n_pairs;
  a.D = c->D;
  a.L = c->L;
  a.smem_surv = 0;
  a.smem_rec_words = 0;
  a.punct_P = c->P;
  a.punct_C = c->punct_C;
  std::memcpy(a.punct_off, c->punct_off, sizeof(a.punct_off));
  std::memcpy(a.punct_pre, c->punct_pre, sizeof(a.punct_pre));
  size_t cnt = 0;
  pbvd_llr_count(c, n_stages, &cnt);
  a.llr_count = (int64_t)cnt;
  a.one = 1u;
  const int64_t grid = ceil_div(p.n_pairs, p.groups);
  if (grid > 0x7fffffff) return PBVD_EINVAL;
  const KernelEntry& e = registry().entries[p.entry];
  PBVD_CUDA(e.launch(a, (int)grid, p.cta, p.smem_bytes, static_cast<cudaStream_t>(stream)));
  return PBVD_OK;
}

size_t pbvd_noalloc_max_survivor_bytes(void) { return kNoAllocSurvivorBytes; }

}  // extern "C"
