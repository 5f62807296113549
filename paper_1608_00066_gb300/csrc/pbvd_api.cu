// Host side of the C ABI declared in include/pbvd.h: argument checks, kernel
// selection, workspace management and launches.  No decoding arithmetic runs
// on the host.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "pbvd.h"
#include "pbvd_internal.h"
#include "pbvd_pm8.h"
#include "pbvd_jit.h"

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
  // entries never move (capacity reserved at start); n_entries publishes how
  // many are complete, so lookups need no lock while codes compiled at run
  // time are appended
  std::vector<KernelEntry> entries;
  std::atomic<size_t> n_entries{0};
  std::vector<int> smem_set;  // max dynamic smem already granted per entry and survivor placement
  std::vector<BatchKernelEntry> batch;
  std::vector<int> batch_smem_set;
  std::vector<StreamKernelEntry> stream;
};

Registry& registry() {
  static Registry reg;
  static std::once_flag once;
  std::call_once(once, [] {
    KernelEntry buf[64];
    int n = 0;
    n += register_k7(buf + n, 64 - n);
    n += register_k7_punctured(buf + n, 64 - n);
    n += register_k9(buf + n, 64 - n);
    n += register_small(buf + n, 64 - n);
    n += register_k7_r3(buf + n, 64 - n);
    // room for codes compiled at run time, so that entries never move
    reg.entries.reserve(4096);
    reg.entries.assign(buf, buf + n);
    reg.smem_set.reserve(2 * 4096);
    reg.smem_set.assign(2 * n, 48 * 1024);
    reg.n_entries.store((size_t)n, std::memory_order_release);
    BatchKernelEntry bb[4];
    const int nb = register_batch(bb, 4);
    reg.batch.assign(bb, bb + nb);
    reg.batch_smem_set.assign(nb, 48 * 1024);
    StreamKernelEntry sb[8];
    const int ns = register_stream(sb, 8);
    reg.stream.assign(sb, sb + ns);
  });
  return reg;
}
std::mutex g_reg_mu;

// var: the instances that honour the traceback / frame variants (selected
// by pbvd_set_mode), else the plain ones.
int find_entry(int K, int R, const uint32_t* gens, int T, bool punct, bool var = false) {
  Registry& reg = registry();
  const size_t count = reg.n_entries.load(std::memory_order_acquire);
  for (size_t i = 0; i < count; ++i) {
    const KernelEntry& e = reg.entries[i];
    if (e.K != K || e.R != R || e.T != T || e.punct != punct) continue;
    if (e.variants != var) continue;
    bool same = true;
    for (int r = 0; r < R; ++r) same = same && (e.gens[r] == gens[r]);
    if (same) return (int)i;
  }
  return -1;
}

int code_has_any_kernel(int K, int R, const uint32_t* gens, bool punct, bool var = false) {
  for (int T = 1; T <= 32; T *= 2)
    if (find_entry(K, R, gens, T, punct, var) >= 0) return 1;
  return 0;
}

// Registers run-time compiled kernels for a code and puncturing with none of
// the kind asked for (plain or variant instances); returns whether the code
// now has such kernels.
int ensure_code_kernels(int K, int R, const uint32_t* gens, bool punct, bool var = false) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  if (code_has_any_kernel(K, R, gens, punct, var)) return 1;
  Registry& reg = registry();
  KernelEntry buf[8];
  const int n = jit_register(K, R, gens, punct, var, buf, 8);
  if (n <= 0 || reg.entries.size() + n > reg.entries.capacity()) return 0;
  for (int i = 0; i < n; ++i) {
    reg.entries.push_back(buf[i]);
    reg.smem_set.push_back(48 * 1024);
    reg.smem_set.push_back(48 * 1024);
  }
  reg.n_entries.store(reg.entries.size(), std::memory_order_release);
  return 1;
}

// Launch of one entry's kernel (built in, or compiled at run time).
int entry_launch(const KernelEntry& e, int smem_surv, const KArgs& a, int grid, int cta, size_t smem,
                 cudaStream_t s) {
  if (e.jit >= 0) {
    const int rc = jit_launch(e.jit, smem_surv ? 1 : 0, a, grid, cta, smem, s);
    if (rc != PBVD_OK) {
      std::lock_guard<std::mutex> lk(g_err_mu);
      std::snprintf(g_last_cuda, sizeof(g_last_cuda), "%s", jit_last_error());
    }
    return rc;
  }
  PBVD_CUDA(e.launch[smem_surv ? 1 : 0](a, grid, cta, smem, s));
  return PBVD_OK;
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
  pbvd_batch* batch;  // work list of the last pbvd_decode_batch led by this context
  // pbvd_decode_host: copy stream, compute lanes, events and device buffers
  int hp_ready;
  cudaStream_t hp_copy;
  cudaStream_t hp_unpack;  // unpacks of packed input, trailing the copies
  cudaEvent_t hp_unp[64];
  cudaStream_t hp_lane[16];
  cudaEvent_t hp_fork;
  cudaEvent_t hp_in[64];
  cudaEvent_t hp_done[16];
  int8_t* hp_llr;
  size_t hp_llr_cap;
  uint8_t* hp_out;
  size_t hp_out_cap;
  uint32_t* hp_surv;
  size_t hp_surv_cap;
  uint32_t* hp_words;    // packed q-bit input of pbvd_decode_host_packed
  size_t hp_words_cap;
  int8_t* pk_vals;       // unpacked values of pbvd_decode_packed
  size_t pk_cap;
  int mode;              // PBVD_MODE_* flags
  int8_t* tb_ext;        // tail-biting: the frame with L wrapped stages on each side
  size_t tb_ext_cap;
  uint32_t* pm8_in;      // pbvd_decode_packed_pm8: gathered values of the quads
  size_t pm8_in_cap;
  uint32_t* pm8_surv;    // pbvd_decode_packed_pm8: survivor records
  size_t pm8_surv_cap;
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

// At most 64 states per thread for codes of up to 64 states, 32 above (the
// 256-state code at four threads per pair, 64 states each, decodes the
// 2^24-bit stream 16% slower than at eight).
int states_max_per_thread(int N) { return N > 64 ? 32 : 64; }

// Automatic kernel configuration.  The throughput form (pbvd_decode) takes
// the fewest threads per pair that still give about 1.5 warps per scheduler:
// fewer threads per pair execute fewer instructions per butterfly (branch
// metrics, transposes, traceback shared by more states), and 1.5 warps
// hide enough latency (K=7 2^24-bit stream at D = 512: two threads per pair
// in 32-thread CTAs 0.2235 ms, four in 64-thread CTAs 0.2309 ms).  The
// pipelined form (pbvd_decode_host, whose runs each end a pair's dependency
// chain after their copy) aims at about 2 warps per scheduler, which gives
// shorter chains (the same stream from host memory: 46.6 against 42.1 Gb/s).
int plan_decode(const pbvd_ctx* c, size_t n_stages, Plan* p, bool pipelined = false) {
  Registry& reg = registry();
  const bool var = c->mode != 0;
  p->n_blocks = ceil_div((int64_t)n_stages, c->D);
  p->n_pairs = ceil_div(p->n_blocks, 2);
  int T = c->cfg.threads_per_pair;
  if (T <= 0) {
    int tmin = 1;
    while (c->N / tmin > states_max_per_thread(c->N)) tmin *= 2;
    // threads for ~1.5 (throughput) or ~2 (pipelined) warps per scheduler
    const int64_t target = (int64_t)c->sm_count * 4 * 32 * (pipelined ? 4 : 3) / 2;
    int64_t want = ceil_div(target, std::max<int64_t>(p->n_pairs, 1));
    T = 1;
    while (T < want && T < 32) T *= 2;
    T = std::max(T, tmin);
    T = std::min(T, std::min(32, c->N / 2));
    while (T > tmin && find_entry(c->K, c->R, c->gens, T, c->P != 0, var) < 0) T /= 2;
    while (T < 32 && find_entry(c->K, c->R, c->gens, T, c->P != 0, var) < 0) T *= 2;
  }
  p->T = T;
  p->entry = find_entry(c->K, c->R, c->gens, T, c->P != 0, var);
  if (p->entry < 0) return PBVD_EUNSUPPORTED;
  const KernelEntry& e = reg.entries[p->entry];
  // survivor records per pair: D + L, rounded up to whole blocks of 8 (the
  // latency kernel stores records eight stages at a time)
  const int64_t jmax = ((int64_t)c->D + c->L + 7) & ~7LL;
  p->rec_words = (int)(((jmax * e.words_per_stage) + 3) & ~3LL);
  int smem = c->cfg.survivors_in_smem;
  if (smem < 0) {
    const int64_t bytes = (int64_t)(p->rec_words + e.scratch_words) * 4;
    smem = (p->n_pairs <= c->sm_count && bytes <= 160 * 1024) ? 1 : 0;
  }
  p->smem_surv = smem;
  int cta = c->cfg.cta_threads;
  // one-warp CTAs at one or two threads per pair (a warp already holds 16
  // or 32 pairs; measured faster than two-warp CTAs there), else 64 threads
  if (cta <= 0) cta = smem ? T : ((!pipelined && T <= 2) ? 32 : std::max(T, 64));
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

int grant_smem(int entry, bool smem_surv, size_t bytes) {
  Registry& reg = registry();
  std::lock_guard<std::mutex> lk(g_reg_mu);
  const int slot = 2 * entry + (smem_surv ? 1 : 0);
  if ((int)bytes <= reg.smem_set[slot]) return PBVD_OK;
  const KernelEntry& e = reg.entries[entry];
  if (e.jit >= 0) {
    const int rc = jit_set_max_smem(e.jit, smem_surv ? 1 : 0, (int)bytes);
    if (rc != PBVD_OK) {
      std::lock_guard<std::mutex> lk2(g_err_mu);
      std::snprintf(g_last_cuda, sizeof(g_last_cuda), "%s", jit_last_error());
      return rc;
    }
  } else {
    PBVD_CUDA(e.set_max_smem[smem_surv ? 1 : 0]((int)bytes));
  }
  reg.smem_set[slot] = (int)bytes;
  return PBVD_OK;
}

}  // namespace


// ------------------------------------------------- host-memory pipeline --

namespace {

constexpr int kHostLanes = 16;
constexpr int kHostMaxSegments = 64;

void host_pipeline_release(pbvd_ctx* c) {
  if (c->hp_ready) {
    cudaStreamDestroy(c->hp_copy);
    cudaStreamDestroy(c->hp_unpack);
    for (int i = 0; i < kHostMaxSegments; ++i) cudaEventDestroy(c->hp_unp[i]);
    for (int l = 0; l < kHostLanes; ++l) {
      cudaStreamDestroy(c->hp_lane[l]);
      cudaEventDestroy(c->hp_done[l]);
    }
    cudaEventDestroy(c->hp_fork);
    for (int i = 0; i < kHostMaxSegments; ++i) cudaEventDestroy(c->hp_in[i]);
    c->hp_ready = 0;
  }
  if (c->hp_llr) cudaFree(c->hp_llr);
  if (c->hp_out) cudaFree(c->hp_out);
  if (c->hp_surv) cudaFree(c->hp_surv);
  if (c->hp_words) cudaFree(c->hp_words);
  if (c->pk_vals) cudaFree(c->pk_vals);
  c->hp_llr = nullptr;
  c->hp_out = nullptr;
  c->hp_surv = nullptr;
  c->hp_words = nullptr;
  c->pk_vals = nullptr;
  c->hp_llr_cap = c->hp_out_cap = c->hp_surv_cap = c->hp_words_cap = c->pk_cap = 0;
}

int host_pipeline_setup(pbvd_ctx* c) {
  if (c->hp_ready) return PBVD_OK;
  // packed input is unpacked on a stream of its own, at the highest
  // priority, so that the copies run back to back and each unpack's CTAs are
  // dispatched ahead of the decode kernels'
  int prio_low = 0, prio_high = 0;
  PBVD_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  PBVD_CUDA(cudaStreamCreateWithFlags(&c->hp_copy, cudaStreamNonBlocking));
  PBVD_CUDA(cudaStreamCreateWithPriority(&c->hp_unpack, cudaStreamNonBlocking, prio_high));
  for (int i = 0; i < kHostMaxSegments; ++i) PBVD_CUDA(cudaEventCreateWithFlags(&c->hp_unp[i], cudaEventDisableTiming));
  for (int l = 0; l < kHostLanes; ++l) {
    PBVD_CUDA(cudaStreamCreateWithFlags(&c->hp_lane[l], cudaStreamNonBlocking));
    PBVD_CUDA(cudaEventCreateWithFlags(&c->hp_done[l], cudaEventDisableTiming));
  }
  PBVD_CUDA(cudaEventCreateWithFlags(&c->hp_fork, cudaEventDisableTiming));
  for (int i = 0; i < kHostMaxSegments; ++i) PBVD_CUDA(cudaEventCreateWithFlags(&c->hp_in[i], cudaEventDisableTiming));
  c->hp_ready = 1;
  return PBVD_OK;
}

// The device address of host memory the kernels may read and write in
// place: page-locked memory mapped into the device's address space
// (cudaHostAlloc / cudaMallocHost / cudaHostRegister under unified
// addressing).  Null for pageable or unknown memory.
void* mapped_host(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

template <class T>
int grow_device(T** p, size_t* cap, size_t bytes) {
  if (bytes <= *cap && *p) return PBVD_OK;
  if (*p) {
    cudaError_t e = cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (e != cudaSuccess) return cuda_fail(e);
  }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes ? bytes : 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e);
  }
  *cap = bytes;
  return PBVD_OK;
}

}  // namespace

// -------------------------------------------------------------- batches --

struct pbvd_batch {
  int device;
  int entry;            // combined kernel
  int grid, cta;
  size_t smem;
  BatchArgs args;
  BatchPair* d_pairs;
  size_t pairs_cap;     // elements
  BatchTile* d_tiles;
  size_t tiles_cap;
  int32_t* d_counter;
  uint32_t* d_surv;
  size_t surv_bytes;
  void* h_stage;        // page-locked staging of the work list (pairs, tiles)
  size_t h_stage_cap;   // bytes
  cudaEvent_t staged;   // the last upload from h_stage
  int staged_pending;
  int single;           // the one code slot of the batch (its own kernel), -1 = mixed
};

namespace {

struct HostPb {
  int item;
  int64_t b;
  int len;    // forward stages f1 - f0 + 1
};

// Forward length of block b of an n-stage stream (Sec. III-A geometry).
int block_len(int64_t n, int D, int L, int64_t b) {
  const int64_t s = b * D - L, e = (b + 1) * D + L;
  const int64_t f0 = s < 0 ? 0 : s;
  const int64_t f1 = (e < n ? e : n) - 1;
  return (int)(f1 - f0 + 1);
}

template <class T>
int grow(T** p, size_t* cap, size_t need) {
  if (need <= *cap && *p) return PBVD_OK;
  if (*p) {
    cudaError_t e = cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (e != cudaSuccess) return cuda_fail(e);
  }
  const size_t n = need > 0 ? need : 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e);
  }
  *cap = n;
  return PBVD_OK;
}

// Builds the work list of a batch into b (created if null): blocks of every
// frame grouped by code slot, sorted by forward length and paired, cut into
// tiles of one CTA's pairs, tiles ordered longest first.  Uploads it on
// 'stream'.
int batch_build(const pbvd_batch_item* items, size_t n_items, void* stream, pbvd_batch* reuse, int reserve_sms,
                pbvd_batch** out) {
  Registry& reg = registry();
  if (reg.batch.empty()) return PBVD_EUNSUPPORTED;
  // the kernel shape: the dense one (entry 1) when a context of the batch
  // asks for its threads-per-pair, else the wide default (entry 0)
  int entry = 0;
  if (reg.batch.size() > 1) {
    for (size_t i = 0; i < n_items; ++i) {
      const pbvd_ctx* c = items[i].ctx;
      if (!c) continue;
      for (int s = 0; s < kBatchSlots; ++s) {
        const BatchKernelEntry& d = reg.batch[1];
        if (d.K[s] == c->K && d.R[s] == c->R && d.punct[s] == (c->P != 0) &&
            c->cfg.threads_per_pair == d.T[s] && reg.batch[0].T[s] != d.T[s])
          entry = 1;
      }
      if (entry == 1) break;
    }
  }
  const BatchKernelEntry& be = reg.batch[entry];
  // map items to code slots; the contexts of a slot must agree on D, L and
  // the puncture pattern
  const pbvd_ctx* slot_ctx[kBatchSlots] = {nullptr, nullptr, nullptr};
  std::vector<int> item_slot(n_items);
  for (size_t i = 0; i < n_items; ++i) {
    const pbvd_batch_item& it = items[i];
    if (!it.ctx || !it.d_llr || !it.d_out || it.n_stages == 0 || it.n_stages > ((size_t)1 << 40))
      return PBVD_EINVAL;
    const pbvd_ctx* c = it.ctx;
    if (c->mode != 0) return PBVD_EUNSUPPORTED;  // the batch kernel decodes the plain scheme
    int slot = -1;
    for (int s = 0; s < kBatchSlots && slot < 0; ++s) {
      if (be.K[s] != c->K || be.R[s] != c->R || be.punct[s] != (c->P != 0)) continue;
      bool same = true;
      for (int r = 0; r < c->R; ++r) same = same && be.gens[s][r] == c->gens[r];
      if (same) slot = s;
    }
    if (slot < 0) return PBVD_EUNSUPPORTED;
    if (!slot_ctx[slot]) {
      slot_ctx[slot] = c;
    } else {
      const pbvd_ctx* r0 = slot_ctx[slot];
      if (r0->D != c->D || r0->L != c->L || r0->P != c->P || r0->device != c->device) return PBVD_EINVAL;
      if (r0->P && std::memcmp(r0->punct_off, c->punct_off, sizeof(c->punct_off)) != 0) return PBVD_EINVAL;
    }
    item_slot[i] = slot;
  }
  const pbvd_ctx* c0 = items[0].ctx;
  int dev = -1;
  PBVD_CUDA(cudaGetDevice(&dev));
  if (dev != c0->device) return PBVD_EINVAL;

  // blocks per slot, longest forward range first (a counting sort on the
  // forward length, stable in item and block order), paired neighbours
  std::vector<const int8_t*> item_end(n_items);
  for (size_t i = 0; i < n_items; ++i) {
    size_t cnt = 0;
    pbvd_llr_count(items[i].ctx, items[i].n_stages, &cnt);
    item_end[i] = items[i].d_llr + cnt;
  }
  std::vector<HostPb> pbs[kBatchSlots];
  std::vector<int64_t> start;
  for (int s = 0; s < kBatchSlots; ++s) {
    if (!slot_ctx[s]) continue;
    const int D = slot_ctx[s]->D, L = slot_ctx[s]->L;
    start.assign((size_t)D + 2 * L + 2, 0);
    int64_t total = 0;
    for (size_t i = 0; i < n_items; ++i) {
      if (item_slot[i] != s) continue;
      const int64_t n = (int64_t)items[i].n_stages, nb = ceil_div(n, D);
      for (int64_t b = 0; b < nb; ++b) ++start[block_len(n, D, L, b)];
      total += nb;
    }
    int64_t acc = 0;
    for (int64_t len = (int64_t)start.size() - 1; len >= 0; --len) {
      const int64_t c = start[len];
      start[len] = acc;
      acc += c;
    }
    pbs[s].resize((size_t)total);
    for (size_t i = 0; i < n_items; ++i) {
      if (item_slot[i] != s) continue;
      const int64_t n = (int64_t)items[i].n_stages, nb = ceil_div(n, D);
      for (int64_t b = 0; b < nb; ++b) {
        const int len = block_len(n, D, L, b);
        pbs[s][(size_t)start[len]++] = {(int)i, b, len};
      }
    }
  }
  const int cta = 64;
  // a batch of one code runs that code's own kernel; mixed batches the
  // combined one
  int single = -1, used = 0;
  for (int s = 0; s < kBatchSlots; ++s)
    if (slot_ctx[s]) {
      ++used;
      single = s;
    }
  if (used != 1) single = -1;
  int Ts[kBatchSlots], scr[kBatchSlots], wps[kBatchSlots];
  for (int s = 0; s < kBatchSlots; ++s) {
    Ts[s] = single >= 0 ? be.single_T[s] : be.T[s];
    scr[s] = single >= 0 ? be.single_scratch_words[s] : be.scratch_words[s];
    wps[s] = single >= 0 ? be.single_words_per_stage[s] : be.words_per_stage[s];
  }
  size_t n_pairs_all = 0;
  for (int s = 0; s < kBatchSlots; ++s) n_pairs_all += (pbs[s].size() + 1) / 2;
  std::vector<BatchTile> tiles;
  std::vector<int64_t> tile_cost;
  for (int s = 0; s < kBatchSlots; ++s) {
    const int64_t np = (int64_t)(pbs[s].size() + 1) / 2;
    if (np == 0) continue;
    const int groups = cta / Ts[s];
    int64_t first_pair = 0;
    for (int q = 0; q < s; ++q) first_pair += (int64_t)(pbs[q].size() + 1) / 2;
    for (int64_t t = 0; t < np; t += groups) {
      BatchTile tl;
      tl.slot = s;
      tl.count = (int)std::min<int64_t>(groups, np - t);
      tl.first = first_pair + t;
      tiles.push_back(tl);
      // pairs are sorted, so the tile's first pair is its longest
      tile_cost.push_back((int64_t)pbs[s][(size_t)(2 * t)].len * (1 << (be.K[s] - 1)) * Ts[s] / 2);
    }
  }
  // longest tiles first for the dynamic tile queue
  std::vector<size_t> order(tiles.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return tile_cost[x] > tile_cost[y]; });

  pbvd_batch* b = reuse;
  if (!b) {
    b = new (std::nothrow) pbvd_batch();
    if (!b) return PBVD_ENOMEM;
    std::memset(b, 0, sizeof(*b));
  }
  b->device = dev;
  b->entry = entry;
  b->cta = cta;
  b->single = single;
  size_t smem = 0;
  int gmax = 0;
  for (int s = 0; s < kBatchSlots; ++s) {
    if (single >= 0 && s != single) continue;
    const int groups = cta / Ts[s];
    smem = std::max(smem, (size_t)groups * scr[s] * 4);
    gmax = std::max(gmax, groups);
  }
  b->smem = smem;
  int rc = PBVD_OK;
  int per_sm = 0;
  if (single < 0) {
    {
      std::lock_guard<std::mutex> lk(g_reg_mu);
      if ((int)smem > reg.batch_smem_set[entry]) {
        cudaError_t e = be.set_max_smem((int)smem);
        if (e != cudaSuccess) return cuda_fail(e);
        reg.batch_smem_set[entry] = (int)smem;
      }
    }
    PBVD_CUDA(be.occupancy(&per_sm, cta, smem));
  } else {
    if (smem > 48 * 1024) PBVD_CUDA(be.single_set_max_smem(single, (int)smem));
    PBVD_CUDA(be.single_occupancy(single, &per_sm, cta, smem));
  }
  if (per_sm < 1) return PBVD_EUNSUPPORTED;
  const int grid_cap = per_sm * std::max(1, c0->sm_count - reserve_sms);
  b->grid = std::max(1, std::min<int>(grid_cap, (int)std::max<size_t>(tiles.size(), 1)));
  const int64_t n_slots = (int64_t)b->grid * gmax;
  // one record slot size for every code of the launch, so that the records
  // of different codes in concurrently running CTAs never overlap
  int rs_max = 0;
  size_t jmax = 0;
  for (int s = 0; s < kBatchSlots; ++s)
    if (slot_ctx[s]) {
      rs_max = std::max(rs_max, wps[s]);
      jmax = std::max(jmax, (size_t)(slot_ctx[s]->D + slot_ctx[s]->L));
    }
  const size_t surv = jmax * (size_t)n_slots * rs_max * 4;
  if ((rc = grow(&b->d_pairs, &b->pairs_cap, n_pairs_all)) != PBVD_OK) return rc;
  if ((rc = grow(&b->d_tiles, &b->tiles_cap, tiles.size())) != PBVD_OK) return rc;
  if (!b->d_counter) PBVD_CUDA(cudaMalloc(&b->d_counter, sizeof(int32_t)));
  size_t surv_words_cap = b->surv_bytes / 4;
  if ((rc = grow(&b->d_surv, &surv_words_cap, (surv + 3) / 4)) != PBVD_OK) return rc;
  b->surv_bytes = surv_words_cap * 4;
  // the work list is written into page-locked staging (once the previous
  // upload from it has left) and uploaded asynchronously
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t pair_bytes = n_pairs_all * sizeof(BatchPair), tile_bytes = tiles.size() * sizeof(BatchTile);
  if (b->staged_pending) {
    PBVD_CUDA(cudaEventSynchronize(b->staged));
    b->staged_pending = 0;
  }
  if (pair_bytes + tile_bytes > b->h_stage_cap) {
    if (b->h_stage) PBVD_CUDA(cudaFreeHost(b->h_stage));
    b->h_stage = nullptr;
    b->h_stage_cap = 0;
    const size_t cap = (pair_bytes + tile_bytes) + (pair_bytes + tile_bytes) / 2 + 4096;
    PBVD_CUDA(cudaHostAlloc(&b->h_stage, cap, cudaHostAllocDefault));
    b->h_stage_cap = cap;
  }
  if (!b->staged) PBVD_CUDA(cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming));
  BatchPair* hp = static_cast<BatchPair*>(b->h_stage);
  BatchTile* ht = reinterpret_cast<BatchTile*>(static_cast<char*>(b->h_stage) + pair_bytes);
  size_t k_pair = 0;
  for (int s = 0; s < kBatchSlots; ++s) {
    const std::vector<HostPb>& v = pbs[s];
    for (size_t k = 0; k < v.size(); k += 2) {
      BatchPair& p = hp[k_pair++];
      for (int h = 0; h < 2; ++h) {
        const HostPb& q = v[k + (k + h < v.size() ? h : 0)];
        const pbvd_batch_item& it = items[q.item];
        p.llr[h] = it.d_llr;
        p.llr_end[h] = item_end[q.item];
        p.out[h] = it.d_out;
        p.n[h] = (int64_t)it.n_stages;
        p.b[h] = q.b;
      }
      p.hasB = (k + 1 < v.size()) ? 1 : 0;
      p.pad = 0;
    }
  }
  for (size_t i = 0; i < order.size(); ++i) ht[i] = tiles[order[i]];
  if (pair_bytes) PBVD_CUDA(cudaMemcpyAsync(b->d_pairs, hp, pair_bytes, cudaMemcpyHostToDevice, st));
  if (tile_bytes) PBVD_CUDA(cudaMemcpyAsync(b->d_tiles, ht, tile_bytes, cudaMemcpyHostToDevice, st));
  PBVD_CUDA(cudaEventRecord(b->staged, st));
  b->staged_pending = 1;
  // kernel arguments
  BatchArgs& a = b->args;
  std::memset(&a, 0, sizeof(a));
  for (int s = 0; s < kBatchSlots; ++s) {
    KArgs& k = a.code[s];
    const pbvd_ctx* c = slot_ctx[s] ? slot_ctx[s] : c0;
    k.D = c->D;
    k.L = c->L;
    k.punct_P = slot_ctx[s] ? c->P : 0;
    k.punct_C = slot_ctx[s] ? c->punct_C : 0;
    std::memcpy(k.punct_off, c->punct_off, sizeof(k.punct_off));
    std::memcpy(k.punct_pre, c->punct_pre, sizeof(k.punct_pre));
    k.surv = b->d_surv;
    k.surv_pairs = n_slots;
    k.surv_rs = rs_max;
    k.smem_surv = 0;
  }
  a.pairs = b->d_pairs;
  a.tiles = b->d_tiles;
  a.ntiles = (int32_t)tiles.size();
  a.gmax = gmax;
  a.counter = b->d_counter;
  *out = b;
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
  if (!code_has_any_kernel(K, R, gens, puncture != nullptr) &&
      !ensure_code_kernels(K, R, gens, puncture != nullptr))
    return PBVD_EUNSUPPORTED;

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
  if (c->batch) pbvd_batch_destroy(c->batch);
  if (c->work || c->hp_ready || c->pm8_surv) cudaDeviceSynchronize();
  if (c->work) cudaFree(c->work);
  if (c->tb_ext) cudaFree(c->tb_ext);
  if (c->pm8_in) cudaFree(c->pm8_in);
  if (c->pm8_surv) cudaFree(c->pm8_surv);
  host_pipeline_release(c);
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
    if (find_entry(c->K, c->R, c->gens, T, c->P != 0) < 0 && find_entry(c->K, c->R, c->gens, T, c->P != 0, true) < 0)
      return PBVD_EUNSUPPORTED;
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

// The decode of pbvd_decode; 'pipelined' selects the automatic configuration
// of host calls (direct access: the kernel's reads of host memory need many
// warps in flight).
static int decode_device(pbvd_ctx* c, const int8_t* d_llr, size_t n_stages, uint8_t* d_out, void* stream,
                         bool pipelined) {
  if (!c || !d_llr || !d_out || n_stages == 0) return PBVD_EINVAL;
  if (n_stages > ((size_t)1 << 40)) return PBVD_EINVAL;
  Plan p;
  int rc = plan_decode(c, n_stages, &p, pipelined);
  if (rc != PBVD_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int8_t* src = d_llr;
  size_t src_count = 0;
  pbvd_llr_count(c, n_stages, &src_count);
  if (c->mode & PBVD_MODE_TAILBITING) {
    // the frame with L stages wrapped around on each side: index e holds
    // stage (e - L) mod n, so every block's window is one contiguous range
    const size_t n = n_stages, L = (size_t)c->L, R = (size_t)c->R;
    rc = grow_device(&c->tb_ext, &c->tb_ext_cap, (n + 2 * L) * R);
    if (rc != PBVD_OK) return rc;
    for (size_t e = 0; e < n + 2 * L;) {
      const size_t stg = (e + n * ((L + n - 1) / n + 1) - L) % n;  // (e - L) mod n
      const size_t len = std::min(n + 2 * L - e, n - stg);
      PBVD_CUDA(cudaMemcpyAsync(c->tb_ext + e * R, d_llr + stg * R, len * R, cudaMemcpyDeviceToDevice, st));
      e += len;
    }
    src = c->tb_ext;
    src_count = (n + 2 * L) * R;
  }
  if (!p.smem_surv) {
    rc = ensure_work(c, p.surv_bytes);
    if (rc != PBVD_OK) return rc;
  }
  rc = grant_smem(p.entry, p.smem_surv != 0, p.smem_bytes);
  if (rc != PBVD_OK) return rc;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.llr = src;
  a.out = d_out;
  a.surv = static_cast<uint32_t*>(c->work);
  a.n = (int64_t)n_stages;
  a.n_blocks = p.n_blocks;
  a.n_pairs = p.n_pairs;
  a.surv_pairs = p.n_pairs;
  a.surv_rs = registry().entries[p.entry].words_per_stage;
  a.D = c->D;
  a.L = c->L;
  a.smem_surv = p.smem_surv;
  a.smem_rec_words = p.smem_surv ? p.rec_words : 0;
  a.punct_P = c->P;
  a.punct_C = c->punct_C;
  std::memcpy(a.punct_off, c->punct_off, sizeof(a.punct_off));
  std::memcpy(a.punct_pre, c->punct_pre, sizeof(a.punct_pre));
  a.llr_count = (int64_t)src_count;
  a.tb_argmin = (c->mode & PBVD_MODE_ARGMIN) ? 1 : 0;
  a.circular = (c->mode & PBVD_MODE_TAILBITING) ? 1 : 0;
  const int64_t grid = ceil_div(p.n_pairs, p.groups);
  if (grid > 0x7fffffff) return PBVD_EINVAL;
  const KernelEntry& e = registry().entries[p.entry];
  return entry_launch(e, p.smem_surv, a, (int)grid, p.cta, p.smem_bytes, st);
}

int pbvd_decode(pbvd_ctx* c, const int8_t* d_llr, size_t n_stages, uint8_t* d_out, void* stream) {
  return decode_device(c, d_llr, n_stages, d_out, stream, false);
}

int pbvd_decode_two_kernel(pbvd_ctx* c, const int8_t* d_llr, size_t n_stages, uint8_t* d_out, void* stream) {
  if (!c || !d_llr || !d_out || n_stages == 0) return PBVD_EINVAL;
  if (n_stages > ((size_t)1 << 40)) return PBVD_EINVAL;
  const int nc = two_kernel_groups(c->K, c->R, c->gens);
  if (nc < 0 || c->P || c->mode) return PBVD_EUNSUPPORTED;
  const int64_t nb = ceil_div((int64_t)n_stages, c->D);
  // SP[D + 2L][N_c][N_t] survivor words
  const size_t sp_bytes = (size_t)(c->D + 2 * c->L) * (size_t)nc * (size_t)nb * 4;
  int rc = ensure_work(c, sp_bytes);
  if (rc != PBVD_OK) return rc;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.llr = d_llr;
  a.out = d_out;
  a.n = (int64_t)n_stages;
  a.n_blocks = nb;
  a.D = c->D;
  a.L = c->L;
  size_t cnt = 0;
  pbvd_llr_count(c, n_stages, &cnt);
  a.llr_count = (int64_t)cnt;
  PBVD_CUDA(two_kernel_launch(c->K, a, static_cast<uint32_t*>(c->work), nb, static_cast<cudaStream_t>(stream)));
  return PBVD_OK;
}

int pbvd_set_mode(pbvd_ctx* c, int flags) {
  if (!c || (flags & ~(PBVD_MODE_ARGMIN | PBVD_MODE_TAILBITING))) return PBVD_EINVAL;
  if ((flags & PBVD_MODE_TAILBITING) && c->P) return PBVD_EUNSUPPORTED;
  // the variant instances are compiled at run time (on their first launch)
  if (flags && !ensure_code_kernels(c->K, c->R, c->gens, c->P != 0, true)) return PBVD_EUNSUPPORTED;
  c->mode = flags;
  return PBVD_OK;
}

int pbvd_get_mode(const pbvd_ctx* c, int* flags) {
  if (!c || !flags) return PBVD_EINVAL;
  *flags = c->mode;
  return PBVD_OK;
}

}  // extern "C"

namespace {

// pbvd_decode_host and pbvd_decode_host_packed: h_in holds int8 soft values
// (q = 0) or q-bit values packed floor(32/q) to a 32-bit word.
int decode_host_impl(pbvd_ctx* c, const void* h_in, int q, size_t n_stages, uint8_t* h_out, int segments,
                     void* stream) {
  if (!c || !h_in || !h_out || n_stages == 0 || segments < -1) return PBVD_EINVAL;
  if (n_stages > ((size_t)1 << 40)) return PBVD_EINVAL;
  if (q < 0 || q > 8) return PBVD_EINVAL;
  const int8_t* h_llr = static_cast<const int8_t*>(h_in);
  const uint32_t* h_words = static_cast<const uint32_t*>(h_in);
  const int64_t per_word = q > 0 ? 32 / q : 1;
  int dev = -1;
  PBVD_CUDA(cudaGetDevice(&dev));
  if (dev != c->device) return PBVD_EINVAL;
  if (segments < 0 && q > 0) return PBVD_EUNSUPPORTED;
  if (c->mode & PBVD_MODE_TAILBITING) return PBVD_EUNSUPPORTED;
  if (segments < 0) {
    // direct access: the kernel reads the soft values from host memory and
    // writes the bits back over the host link itself, with no staging copy
    const int8_t* d_in = static_cast<const int8_t*>(mapped_host(h_llr));
    uint8_t* d_o = static_cast<uint8_t*>(mapped_host(h_out));
    if (!d_in || !d_o) return PBVD_EINVAL;
    return decode_device(c, d_in, n_stages, d_o, stream, true);
  }
  // the kernel configuration pbvd_decode would use, survivors in global
  // memory (one workspace slice per compute lane)
  pbvd_ctx cc = *c;
  cc.cfg.survivors_in_smem = 0;
  Plan p;
  int rc = plan_decode(&cc, n_stages, &p, true);
  if (rc != PBVD_OK) return rc;
  const int64_t nb = p.n_blocks;
  // runs of whole pairs of blocks; automatic: up to 6 runs (fewer for packed
  // input, below) of at least 1024 blocks.  A run's decode takes at least the dependency chain of one pair
  // (about half the whole stream's decode time for 4 threads per pair), so
  // more, shorter runs start sooner but end no sooner; runs with a
  // different kernel configuration (a shorter chain) slowed the whole call
  // down, the kernels sharing the SMs badly.
  // Packed input crosses the link in a fraction of the time, and its runs
  // also wait for their unpacking: fewer runs (measured on the 2^24-bit K=7
  // stream: 2 runs best for q <= 3, 4 for q >= 4, against 6 for int8 input).
  const int64_t auto_runs = q == 0 ? 6 : (q <= 3 ? 2 : 4);
  int64_t want = segments > 0 ? segments : std::max<int64_t>(1, std::min<int64_t>(auto_runs, nb / 1024));
  want = std::min<int64_t>(std::min<int64_t>(want, kHostMaxSegments), nb);
  int64_t bps = ceil_div(nb, want);
  bps += bps & 1;  // whole pairs per run
  struct Run {
    int64_t b0, b1;
  };
  std::vector<Run> runs;
  for (int64_t b = 0; b < nb; b += bps) runs.push_back({b, std::min(nb, b + bps)});
  const int S = (int)runs.size();
  if (S > kHostMaxSegments) return PBVD_EINVAL;
  const KernelEntry& e = registry().entries[p.entry];
  const int64_t jmax = ((int64_t)c->D + c->L + 7) & ~7LL;
  const size_t slice_words = (size_t)jmax * (size_t)(bps / 2) * e.words_per_stage;
  size_t llr_bytes = 0;
  pbvd_llr_count(c, n_stages, &llr_bytes);
  const size_t out_bytes = (n_stages + 7) / 8;
  rc = host_pipeline_setup(c);
  if (rc != PBVD_OK) return rc;
  rc = grow_device(&c->hp_llr, &c->hp_llr_cap, llr_bytes);
  if (rc != PBVD_OK) return rc;
  rc = grow_device(&c->hp_out, &c->hp_out_cap, out_bytes);
  if (rc != PBVD_OK) return rc;
  rc = grow_device(&c->hp_surv, &c->hp_surv_cap, (size_t)kHostLanes * slice_words * 4);
  if (rc != PBVD_OK) return rc;
  const size_t n_words = q > 0 ? (size_t)((llr_bytes + per_word - 1) / per_word) : 0;
  if (q > 0) {
    rc = grow_device(&c->hp_words, &c->hp_words_cap, n_words * 4);
    if (rc != PBVD_OK) return rc;
  }
  rc = grant_smem(p.entry, false, p.smem_bytes);
  if (rc != PBVD_OK) return rc;

  cudaStream_t user = static_cast<cudaStream_t>(stream);
  PBVD_CUDA(cudaEventRecord(c->hp_fork, user));
  PBVD_CUDA(cudaStreamWaitEvent(c->hp_copy, c->hp_fork, 0));
  for (int l = 0; l < kHostLanes; ++l) PBVD_CUDA(cudaStreamWaitEvent(c->hp_lane[l], c->hp_fork, 0));
  // soft values in order on one copy stream: copy i ends L stages into run
  // i + 1 (the last stage run i's blocks read), so run i waits for copy i only
  auto copy_edge = [&](int i) -> size_t {
    if (i <= 0) return 0;
    if (i >= S) return n_stages;
    return std::min(n_stages, (size_t)(runs[i].b0 * c->D + c->L));
  };
  for (int i = 0; i < S; ++i) {
    const size_t s0 = copy_edge(i);
    const size_t s1 = copy_edge(i + 1);
    size_t v0 = 0, v1 = 0;
    pbvd_llr_count(c, s0, &v0);
    pbvd_llr_count(c, s1, &v1);
    if (v1 > v0 && q == 0) {
      PBVD_CUDA(cudaMemcpyAsync(c->hp_llr + v0, h_llr + v0, v1 - v0, cudaMemcpyHostToDevice, c->hp_copy));
    } else if (v1 > v0) {
      // the words holding values [v0, v1) (a word shared with the previous
      // copy is copied again; same bytes, same stream), then their values
      const size_t w0 = v0 / per_word, w1 = std::min(n_words, (v1 + per_word - 1) / per_word);
      PBVD_CUDA(cudaMemcpyAsync(c->hp_words + w0, h_words + w0, (w1 - w0) * 4, cudaMemcpyHostToDevice,
                                c->hp_copy));
    }
    PBVD_CUDA(cudaEventRecord(c->hp_in[i], c->hp_copy));
    if (q > 0) {
      // values [v0, v1) once their words have arrived (in order, so run i
      // finds every value before v1 unpacked)
      PBVD_CUDA(cudaStreamWaitEvent(c->hp_unpack, c->hp_in[i], 0));
      if (v1 > v0) PBVD_CUDA(launch_unpack(q, c->hp_words, (int64_t)v0, (int64_t)v1, c->hp_llr, c->hp_unpack));
      PBVD_CUDA(cudaEventRecord(c->hp_unp[i], c->hp_unpack));
    }
  }
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.llr = c->hp_llr;
  a.out = c->hp_out;
  a.n = (int64_t)n_stages;
  a.surv_rs = e.words_per_stage;
  a.D = c->D;
  a.L = c->L;
  a.smem_surv = 0;
  a.smem_rec_words = 0;
  a.punct_P = c->P;
  a.punct_C = c->punct_C;
  std::memcpy(a.punct_off, c->punct_off, sizeof(a.punct_off));
  std::memcpy(a.punct_pre, c->punct_pre, sizeof(a.punct_pre));
  a.llr_count = (int64_t)llr_bytes;
  a.tb_argmin = (c->mode & PBVD_MODE_ARGMIN) ? 1 : 0;
  for (int i = 0; i < S; ++i) {
    const int l = i % kHostLanes;
    cudaStream_t st = c->hp_lane[l];
    PBVD_CUDA(cudaStreamWaitEvent(st, q > 0 ? c->hp_unp[i] : c->hp_in[i], 0));
    const Run& r = runs[i];
    a.b_first = r.b0;
    a.n_blocks = r.b1;
    a.n_pairs = ceil_div(r.b1 - r.b0, 2);
    a.surv = c->hp_surv + (size_t)l * slice_words;
    a.surv_pairs = a.n_pairs;
    const int64_t grid = ceil_div(a.n_pairs, p.groups);
    rc = entry_launch(e, 0, a, (int)grid, p.cta, p.smem_bytes, st);
    if (rc != PBVD_OK) return rc;
    const size_t o0 = (size_t)(r.b0 * c->D / 8);
    const size_t o1 = (std::min(n_stages, (size_t)(r.b1 * c->D)) + 7) / 8;
    PBVD_CUDA(cudaMemcpyAsync(h_out + o0, c->hp_out + o0, o1 - o0, cudaMemcpyDeviceToHost, st));
  }
  for (int l = 0; l < kHostLanes; ++l) {
    PBVD_CUDA(cudaEventRecord(c->hp_done[l], c->hp_lane[l]));
    PBVD_CUDA(cudaStreamWaitEvent(user, c->hp_done[l], 0));
  }
  return PBVD_OK;
}

}  // namespace

extern "C" {

int pbvd_decode_host(pbvd_ctx* c, const int8_t* h_llr, size_t n_stages, uint8_t* h_out, int segments,
                     void* stream) {
  return decode_host_impl(c, h_llr, 0, n_stages, h_out, segments, stream);
}

int pbvd_decode_host_packed(pbvd_ctx* c, const uint32_t* h_words, int q, size_t n_stages, uint8_t* h_out,
                            int segments, void* stream) {
  if (q < 1 || q > 8 || segments < 0) return PBVD_EINVAL;
  return decode_host_impl(c, h_words, q, n_stages, h_out, segments, stream);
}

int pbvd_decode_packed(pbvd_ctx* c, const uint32_t* d_words, int q, size_t n_stages, uint8_t* d_out,
                       void* stream) {
  if (!c || !d_words || !d_out || n_stages == 0 || q < 1 || q > 8) return PBVD_EINVAL;
  if (n_stages > ((size_t)1 << 40)) return PBVD_EINVAL;
  size_t count = 0;
  pbvd_llr_count(c, n_stages, &count);
  int rc = grow_device(&c->pk_vals, &c->pk_cap, count + 16);
  if (rc != PBVD_OK) return rc;
  PBVD_CUDA(launch_unpack(q, d_words, 0, (int64_t)count, c->pk_vals, static_cast<cudaStream_t>(stream)));
  return pbvd_decode(c, c->pk_vals, n_stages, d_out, stream);
}

int pbvd_decode_packed_pm8(pbvd_ctx* c, const uint32_t* d_words, int q, size_t n_stages, uint8_t* d_out,
                           void* stream) {
  if (!c || !d_words || !d_out || n_stages == 0 || q < 1 || q > 8) return PBVD_EINVAL;
  if (n_stages > ((size_t)1 << 40)) return PBVD_EINVAL;
  if (c->P != 0 || c->mode != 0) return PBVD_EUNSUPPORTED;
  pbvd::Pm8Plan plan;
  int64_t I = 0, nquads = 0;
  size_t in_words = 0, surv_words = 0;
  pbvd::pm8_sizes(c->K, c->R, (int64_t)n_stages, c->D, c->L, &I, &nquads, &in_words, &surv_words);
  // threads per four blocks: 1 or 2 when the context's threads_per_pair says
  // so; otherwise two (where built) while one thread per four blocks would
  // leave fewer than two warps per SM (measured: 2^24-bit K=7 stream at
  // D = 512, 8,193 quads: 0.55 against 0.84 ms; at D = 256: 0.57 against
  // 0.50 ms)
  int lanes = c->cfg.threads_per_pair;
  if (lanes != 1 && lanes != 2) {
    pbvd::Pm8Plan two;
    lanes = (nquads < (int64_t)64 * c->sm_count && pbvd::pm8_plan(c->K, c->R, c->gens, q, 2, &two) == 0) ? 2 : 1;
  }
  if (pbvd::pm8_plan(c->K, c->R, c->gens, q, lanes, &plan) != 0) return PBVD_EUNSUPPORTED;
  if ((2 * nquads + 31) / 32 > INT32_MAX) return PBVD_EINVAL;
  int rc = grow_device(&c->pm8_in, &c->pm8_in_cap, in_words * 4);
  if (rc != PBVD_OK) return rc;
  rc = grow_device(&c->pm8_surv, &c->pm8_surv_cap, surv_words * 4);
  if (rc != PBVD_OK) return rc;
  PBVD_CUDA(pbvd::pm8_launch(plan, c->K, c->R, d_words, (int64_t)n_stages, c->D, c->L, c->pm8_in, c->pm8_surv,
                             d_out, static_cast<cudaStream_t>(stream)));
  return PBVD_OK;
}

int pbvd_decode_batch(const pbvd_batch_item* items, size_t n_items, void* stream) {
  if (!items && n_items) return PBVD_EINVAL;
  if (n_items == 0) return PBVD_OK;
  if (!items[0].ctx) return PBVD_EINVAL;
  pbvd_ctx* lead = items[0].ctx;
  int rc = batch_build(items, n_items, stream, lead->batch ? lead->batch : nullptr, 0, &lead->batch);
  if (rc != PBVD_OK) return rc;
  return pbvd_batch_run(lead->batch, stream);
}

int pbvd_batch_prepare(pbvd_batch** out, const pbvd_batch_item* items, size_t n_items, void* stream) {
  if (!out || (!items && n_items) || n_items == 0) return PBVD_EINVAL;
  *out = nullptr;
  pbvd_batch* b = nullptr;
  int rc = batch_build(items, n_items, stream, nullptr, 0, &b);
  if (rc != PBVD_OK) {
    if (b) pbvd_batch_destroy(b);
    return rc;
  }
  *out = b;
  return PBVD_OK;
}

int pbvd_batch_update(pbvd_batch* b, const pbvd_batch_item* items, size_t n_items, int reserve_sms, void* stream) {
  if (!b || !items || n_items == 0 || reserve_sms < 0) return PBVD_EINVAL;
  pbvd_batch* same = b;
  return batch_build(items, n_items, stream, b, reserve_sms, &same);
}

int pbvd_batch_run(pbvd_batch* b, void* stream) {
  if (!b) return PBVD_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (b->args.ntiles == 0) return PBVD_OK;
  PBVD_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(int32_t), st));
  const BatchKernelEntry& be = registry().batch[b->entry];
  if (b->single >= 0)
    PBVD_CUDA(be.single_launch(b->args, b->single, b->grid, b->cta, b->smem, st));
  else
    PBVD_CUDA(be.launch(b->args, b->grid, b->cta, b->smem, st));
  return PBVD_OK;
}

void pbvd_batch_destroy(pbvd_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->d_pairs) cudaFree(b->d_pairs);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->d_surv) cudaFree(b->d_surv);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  if (b->staged) cudaEventDestroy(b->staged);
  delete b;
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
// first call outside any stream capture.  The looked-up address is kept for
// the life of the process, so the device must not be reset
// (cudaDeviceReset) while the library is in use.  All calls share the array and it
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
  if (c->mode & PBVD_MODE_TAILBITING) return PBVD_EUNSUPPORTED;  // needs the wrapped copy of the frame
  // survivor bits in shared memory (when the context's configuration picks
  // that placement; it allocates nothing) or in the fixed array
  pbvd_ctx cc = *c;
  Plan p;
  int rc = plan_decode(&cc, n_stages, &p);
  if (rc != PBVD_OK) return rc;
  if (!p.smem_surv) {
    cc.cfg.survivors_in_smem = 0;
    rc = plan_decode(&cc, n_stages, &p);
    if (rc != PBVD_OK) return rc;
  }
  // with an automatic thread count, fall back to fewer threads per pair
  // (smaller survivor records) until the survivor bits fit the array
  while (!p.smem_surv && c->cfg.threads_per_pair == 0 && p.surv_bytes > kNoAllocSurvivorBytes && p.T > 1) {
    cc.cfg.threads_per_pair = p.T / 2;
    if (find_entry(c->K, c->R, c->gens, cc.cfg.threads_per_pair, c->P != 0, c->mode != 0) < 0) break;
    rc = plan_decode(&cc, n_stages, &p);
    if (rc != PBVD_OK) return rc;
  }
  if (!p.smem_surv && p.surv_bytes > kNoAllocSurvivorBytes) return PBVD_EINVAL;
  // a kernel compiled at run time must be loaded already: loading it
  // allocates device memory for its code
  {
    const KernelEntry& ej = registry().entries[p.entry];
    if (ej.jit >= 0 && !jit_loaded(ej.jit, p.smem_surv ? 1 : 0)) return PBVD_EUNSUPPORTED;
  }
  uint32_t* surv = nullptr;
  rc = noalloc_survivors(dev, &surv);
  if (rc != PBVD_OK) return rc;
  rc = grant_smem(p.entry, p.smem_surv != 0, p.smem_bytes);
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
  a.surv_rs = registry().entries[p.entry].words_per_stage;
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
  a.tb_argmin = (c->mode & PBVD_MODE_ARGMIN) ? 1 : 0;
  const int64_t grid = ceil_div(p.n_pairs, p.groups);
  if (grid > 0x7fffffff) return PBVD_EINVAL;
  const KernelEntry& e = registry().entries[p.entry];
  return entry_launch(e, p.smem_surv, a, (int)grid, p.cta, p.smem_bytes, static_cast<cudaStream_t>(stream));
}

size_t pbvd_noalloc_max_survivor_bytes(void) { return kNoAllocSurvivorBytes; }

}  // extern "C"

// ---------------------------------------------------------------- tuning --

extern "C" {

int pbvd_autotune(pbvd_ctx* c, const int8_t* d_llr, size_t n_stages, uint8_t* d_out, void* stream, int reps,
                  pbvd_config* best_cfg, float* best_ms) {
  if (!c || !d_llr || !d_out || n_stages == 0) return PBVD_EINVAL;
  if (reps < 1) reps = 3;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const pbvd_config saved = c->cfg;
  cudaEvent_t e0, e1;
  PBVD_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce);
  }
  pbvd_config best = saved;
  float best_t = -1.0f;
  int rc = PBVD_OK;
  for (int T = 1; T <= 32 && rc == PBVD_OK; T *= 2) {
    if (find_entry(c->K, c->R, c->gens, T, c->P != 0, c->mode != 0) < 0) continue;
    for (int cta : {32, 64, 128, 256}) {
      if (cta % T) continue;
      for (int smem = 0; smem <= 1; ++smem) {
        c->cfg.threads_per_pair = T;
        c->cfg.cta_threads = cta;
        c->cfg.survivors_in_smem = smem;
        Plan p;
        if (plan_decode(c, n_stages, &p) != PBVD_OK) continue;
        // skip shapes that cannot fill the GPU with one pair per group
        if (smem && p.n_pairs > 4 * c->sm_count) continue;
        if (pbvd_decode(c, d_llr, n_stages, d_out, stream) != PBVD_OK) continue;  // warm-up
        float tot = 0.0f;
        for (int r = 0; r < reps && rc == PBVD_OK; ++r) {
          cudaEventRecord(e0, st);
          rc = pbvd_decode(c, d_llr, n_stages, d_out, stream);
          cudaEventRecord(e1, st);
          ce = cudaEventSynchronize(e1);
          if (ce != cudaSuccess) rc = cuda_fail(ce);
          float ms = 0.0f;
          cudaEventElapsedTime(&ms, e0, e1);
          tot += ms;
        }
        const float t = tot / reps;
        if (rc == PBVD_OK && (best_t < 0.0f || t < best_t)) {
          best_t = t;
          best = c->cfg;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PBVD_OK || best_t < 0.0f) {
    c->cfg = saved;
    return rc != PBVD_OK ? rc : PBVD_EUNSUPPORTED;
  }
  c->cfg = best;
  if (best_cfg) *best_cfg = best;
  if (best_ms) *best_ms = best_t;
  return PBVD_OK;
}

}  // extern "C"

// -------------------------------------------------------------- streams --

struct pbvd_stream {
  pbvd_ctx* ctx;
  int entry;
  int P, R, H;
  size_t max_push;
  int64_t t;          // stages decoded (forward)
  int64_t released;   // stages whose bits are final
  int carry;          // stages held back (< P)
  int closed;
  uint8_t* d_out;
  size_t out_cap;     // stages
  uint32_t* d_pm;
  uint32_t* d_ring;
  int8_t* d_carry;
};

namespace {

int find_stream_entry(const pbvd_ctx* c) {
  Registry& reg = registry();
  for (size_t i = 0; i < reg.stream.size(); ++i) {
    const StreamKernelEntry& e = reg.stream[i];
    if (e.K != c->K || e.R != c->R) continue;
    bool same = true;
    for (int r = 0; r < c->R; ++r) same = same && e.gens[r] == c->gens[r];
    if (same) return (int)i;
  }
  return -1;
}

}  // namespace

extern "C" {

int pbvd_stream_open(pbvd_stream** out, pbvd_ctx* c, size_t max_push, uint8_t* d_out, size_t out_capacity) {
  if (!out) return PBVD_EINVAL;
  *out = nullptr;
  if (!c || !d_out || max_push == 0 || max_push > ((size_t)1 << 24) || out_capacity == 0) return PBVD_EINVAL;
  if (c->P || c->mode != 0) return PBVD_EUNSUPPORTED;  // streams: the carried-metric window form only
  const int entry = find_stream_entry(c);
  if (entry < 0) return PBVD_EUNSUPPORTED;
  const StreamKernelEntry& e = registry().stream[entry];
  pbvd_stream* s = new (std::nothrow) pbvd_stream();
  if (!s) return PBVD_ENOMEM;
  std::memset(s, 0, sizeof(*s));
  s->ctx = c;
  s->entry = entry;
  s->P = e.P;
  s->R = c->R;
  s->max_push = max_push;
  // records of the oldest unreleased stage up to the last stage of a push,
  // rounded up to whole blocks of eight stages with one block to spare
  s->H = (int)((max_push + c->D + c->L + 2 * e.P + 8 + 7) & ~(size_t)7);
  s->d_out = d_out;
  s->out_cap = out_capacity;
  // known start: S_0 at 0, every other state at 8192 (lane A)
  std::vector<uint32_t> pm0(c->N, 8192u);
  pm0[0] = 0u;
  cudaError_t ce = cudaMalloc(&s->d_pm, sizeof(uint32_t) * c->N);
  if (ce == cudaSuccess) ce = cudaMalloc(&s->d_ring, (size_t)s->H * e.words_per_stage * sizeof(uint32_t));
  if (ce == cudaSuccess) ce = cudaMalloc(&s->d_carry, (size_t)e.P * c->R);
  if (ce == cudaSuccess) ce = cudaMemcpy(s->d_pm, pm0.data(), sizeof(uint32_t) * c->N, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    pbvd_stream_destroy(s);
    return cuda_fail(ce);
  }
  *out = s;
  return PBVD_OK;
}

void pbvd_stream_destroy(pbvd_stream* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  if (s->d_pm) cudaFree(s->d_pm);
  if (s->d_ring) cudaFree(s->d_ring);
  if (s->d_carry) cudaFree(s->d_carry);
  delete s;
}

int64_t pbvd_stream_released(const pbvd_stream* s) { return s ? s->released : -1; }

int pbvd_stream_metrics(const pbvd_stream* s, int64_t* stages, int32_t* h_metrics, void* stream) {
  if (!s || !stages || !h_metrics) return PBVD_EINVAL;
  const int N = s->ctx->N;
  std::vector<uint32_t> w((size_t)N);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PBVD_CUDA(cudaMemcpyAsync(w.data(), s->d_pm, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost, st));
  PBVD_CUDA(cudaStreamSynchronize(st));
  for (int u = 0; u < N; ++u) h_metrics[u] = (int32_t)(w[u] & 0xFFFFu);  // lane A, natural state order
  *stages = s->t;
  return PBVD_OK;
}

int pbvd_stream_push_many(pbvd_stream* const* ss, const int8_t* const* d_llr, const size_t* n_stages,
                          size_t count, int close, void* stream) {
  if (!ss || count == 0) return PBVD_EINVAL;
  const int entry = ss[0] ? ss[0]->entry : -1;
  for (size_t i = 0; i < count; ++i) {
    const pbvd_stream* s = ss[i];
    if (!s || s->closed || s->entry != entry) return PBVD_EINVAL;
    for (size_t j = 0; j < i; ++j)
      if (ss[j] == s) return PBVD_EINVAL;
    const size_t n = n_stages ? n_stages[i] : 0;
    if (n > s->max_push || (n && (!d_llr || !d_llr[i]))) return PBVD_EINVAL;
    if ((size_t)(s->t + s->carry) + n > s->out_cap) return PBVD_EINVAL;
  }
  const StreamKernelEntry& e = registry().stream[entry];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  static thread_local StreamLaunch p;
  for (size_t base = 0; base < count; base += kStreamsPerLaunch) {
    const int m = (int)std::min<size_t>(kStreamsPerLaunch, count - base);
    p.count = m;
    for (int i = 0; i < m; ++i) {
      const pbvd_stream* s = ss[base + i];
      const size_t n = n_stages ? n_stages[base + i] : 0;
      StreamDev& d = p.d[i];
      d.pm = s->d_pm;
      d.ring = s->d_ring;
      d.carry = s->d_carry;
      d.llr = n ? d_llr[base + i] : nullptr;
      d.out = s->d_out;
      d.t0 = s->t;
      d.released = s->released;
      d.ncarry = s->carry;
      d.nnew = (int32_t)n;
      d.final_ = close ? 1 : 0;
      d.H = s->H;
      d.D = s->ctx->D;
      d.L = s->ctx->L;
    }
    PBVD_CUDA(e.launch(p, st));
  }
  // host bookkeeping mirrors the kernel: whole periods decoded, segments
  // released once their trigger stage exists, everything at close
  for (size_t i = 0; i < count; ++i) {
    pbvd_stream* s = ss[i];
    const int64_t nst = s->carry + (int64_t)(n_stages ? n_stages[i] : 0);
    const int64_t nproc = close ? nst : (nst / s->P) * s->P;
    const int64_t tend = s->t + nproc;
    const int64_t D = s->ctx->D, L = s->ctx->L;
    int64_t nseg = 0;
    if (tend >= s->released + D + L) nseg = (tend - L - s->released) / D;
    s->t = tend;
    s->released = close ? tend : s->released + nseg * D;
    s->carry = (int)(nst - nproc);
    if (close) s->closed = 1;
  }
  return PBVD_OK;
}

int pbvd_stream_push(pbvd_stream* s, const int8_t* d_llr, size_t n_stages, void* stream) {
  return pbvd_stream_push_many(&s, &d_llr, &n_stages, 1, 0, stream);
}

int pbvd_stream_close(pbvd_stream* s, void* stream) {
  return pbvd_stream_push_many(&s, nullptr, nullptr, 1, 1, stream);
}

}  // extern "C"
