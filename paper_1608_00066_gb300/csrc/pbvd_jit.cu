// Kernels for codes chosen at run time.
//
// The paper's decoder serves any (R,1,K) code (Sec. III-B: the branch-metric
// groups of Eqs. (3)-(6) follow from the generators), and pbvd_create takes
// the generators as arguments.  The library carries compiled kernels for the
// codes of the paper's experiments and of the benchmark workloads; for any
// other code it compiles the same kernel template (pbvd_device.cuh) for that
// code's generators with NVRTC, the first time a launch needs it, and loads
// the result with the CUDA runtime's library API.  The generators then become
// compile-time constants again: the codeword relabelling per register, the
// complement symmetry of the branch metrics (when every generator taps the
// oldest cell) and the decision constants are resolved by the compiler exactly
// as for the built-in codes, so a code chosen at run time decodes at the speed
// and with the bits of a built-in one.
//
// The decoding variants (argmin traceback start, tail-biting frames) are
// compiled the same way for every code, built-in ones included, when a
// context first selects them, so that the built-in plain kernels carry none
// of their code.
//
// libnvrtc is opened with dlopen when the first such code is created; without
// it pbvd_create keeps returning PBVD_EUNSUPPORTED for those codes.  The kernel
// sources are embedded in the library at build time (pbvd_jit_src.inc), so
// nothing is read from disk.
#include <dlfcn.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>
#include <nvrtc.h>

#include "pbvd.h"
#include "pbvd_device.cuh"
#include "pbvd_internal.h"
#include "pbvd_jit.h"

namespace pbvd {
namespace {

#include "pbvd_jit_src.inc"  // kJitNumHeaders, kJitHeaderNames[], kJitHeaders[]

// ------------------------------------------------------------ libnvrtc --

struct Nvrtc {
  bool ok = false;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&nvrtcAddNameExpression) add_name = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcGetLoweredName) lowered = nullptr;
};

Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
    for (const char* env : {"CUDA_HOME", "CUDA_PATH"}) {
      const char* root = std::getenv(env);
      if (root && *root) names.push_back(std::string(root) + "/lib64/libnvrtc.so.13");
    }
    names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
    void* h = nullptr;
    for (const std::string& nm : names)
      if ((h = dlopen(nm.c_str(), RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) return;
    bool all = true;
    auto sym = [&](auto& fn, const char* name) {
      fn = reinterpret_cast<std::remove_reference_t<decltype(fn)>>(dlsym(h, name));
      all = all && fn != nullptr;
    };
    sym(n.create, "nvrtcCreateProgram");
    sym(n.destroy, "nvrtcDestroyProgram");
    sym(n.add_name, "nvrtcAddNameExpression");
    sym(n.compile, "nvrtcCompileProgram");
    sym(n.log_size, "nvrtcGetProgramLogSize");
    sym(n.log, "nvrtcGetProgramLog");
    sym(n.cubin_size, "nvrtcGetCUBINSize");
    sym(n.cubin, "nvrtcGetCUBIN");
    sym(n.lowered, "nvrtcGetLoweredName");
    n.ok = all;
  });
  return n;
}

// ------------------------------------------------- shapes on the host --

// Record and scratch sizes depend on K, R and T only (not on the generators),
// so the host reads them off a representative code of the same K and R.
template <int K, int R>
using RepCode = Code<K, (1u << (K - 1)) | 1u, (1u << (K - 1)) | 1u, R == 3 ? ((1u << (K - 1)) | 1u) : 0u>;

template <int K, int R, int T>
void shape_of(int* words_per_stage, int* scratch_words) {
  constexpr int N = 1 << (K - 1);
  if constexpr (T <= N / 2 && N / T <= 64) {
    *words_per_stage = record_words_per_stage<RepCode<K, R>, T>();
    *scratch_words = scratch_words_per_group<RepCode<K, R>, T>();
  } else {
    *words_per_stage = 0;
    *scratch_words = 0;
  }
}

template <int K, int R>
void shape_kr(int T, int* w, int* s) {
  switch (T) {
    case 1: shape_of<K, R, 1>(w, s); break;
    case 2: shape_of<K, R, 2>(w, s); break;
    case 4: shape_of<K, R, 4>(w, s); break;
    case 8: shape_of<K, R, 8>(w, s); break;
    case 16: shape_of<K, R, 16>(w, s); break;
    case 32: shape_of<K, R, 32>(w, s); break;
    default: *w = 0; *s = 0;
  }
}

template <int R>
void shape_r(int K, int T, int* w, int* s) {
  switch (K) {
    case 3: shape_kr<3, R>(T, w, s); break;
    case 4: shape_kr<4, R>(T, w, s); break;
    case 5: shape_kr<5, R>(T, w, s); break;
    case 6: shape_kr<6, R>(T, w, s); break;
    case 7: shape_kr<7, R>(T, w, s); break;
    case 8: shape_kr<8, R>(T, w, s); break;
    case 9: shape_kr<9, R>(T, w, s); break;
    default: *w = 0; *s = 0;
  }
}

void shape(int K, int R, int T, int* w, int* s) {
  if (R == 2) shape_r<2>(K, T, w, s);
  else if (R == 3) shape_r<3>(K, T, w, s);
  else *w = *s = 0;
}

// ------------------------------------------------------- kernel table --

// One (code, T, punctured) instance; its two survivor placements are
// compiled separately, each on first use.
struct JitKernel {
  int K, R, T;
  uint32_t gens[3];
  bool punct;
  bool var;  // the instance honouring the traceback / frame variants
  cudaLibrary_t lib[2] = {nullptr, nullptr};
  cudaKernel_t fn[2] = {nullptr, nullptr};
  int smem_granted[2] = {48 * 1024, 48 * 1024};
};

std::mutex g_jit_mu;
std::vector<JitKernel*> g_jit;   // never shrinks; entries keep their index
char g_jit_err[1024] = "no error";

void set_err(const std::string& m) {
  std::snprintf(g_jit_err, sizeof(g_jit_err), "%s", m.c_str());
}

std::string kernel_name(const JitKernel& k, int smem) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "pbvd::pbvd_decode_kernel<pbvd::Code<%d, %uu, %uu, %uu>, %d, %s, %s, %s>", k.K,
                k.gens[0], k.gens[1], k.gens[2], k.T, k.punct ? "true" : "false", smem ? "true" : "false",
                k.var ? "true" : "false");
  return buf;
}

// Compiles and loads one placement of kernel k (g_jit_mu held).
int compile(JitKernel& k, int smem) {
  Nvrtc& rt = nvrtc();
  if (!rt.ok) {
    set_err("libnvrtc not found");
    return PBVD_EUNSUPPORTED;
  }
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    set_err("no CUDA device for run-time compilation");
    return PBVD_ECUDA;
  }
  const std::string name = kernel_name(k, smem);
  const std::string src = "#include \"pbvd_device.cuh\"\ntemplate __global__ void " + name +
                          "(const pbvd::KArgs);\n";
  nvrtcProgram prog = nullptr;
  if (rt.create(&prog, src.c_str(), "pbvd_jit_instance.cu", kJitNumHeaders, kJitHeaders, kJitHeaderNames) !=
      NVRTC_SUCCESS) {
    set_err("nvrtcCreateProgram failed");
    return PBVD_EUNSUPPORTED;
  }
  char arch[32];
  std::snprintf(arch, sizeof(arch), "-arch=sm_%d%d%s", major, minor, major >= 9 ? "a" : "");
  const char* opts[] = {arch, "-std=c++17", "-default-device", "-lineinfo"};
  rt.add_name(prog, name.c_str());
  const nvrtcResult cr = rt.compile(prog, 4, opts);
  if (cr != NVRTC_SUCCESS) {
    size_t n = 0;
    rt.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) rt.log(prog, &log[0]);
    set_err("run-time compilation of " + name + " failed: " + log.substr(0, 700));
    rt.destroy(&prog);
    return PBVD_EUNSUPPORTED;
  }
  size_t cubin_bytes = 0;
  rt.cubin_size(prog, &cubin_bytes);
  std::vector<char> cubin(cubin_bytes);
  rt.cubin(prog, cubin.data());
  const char* lowered = nullptr;
  rt.lowered(prog, name.c_str(), &lowered);
  const std::string low = lowered ? lowered : "";
  rt.destroy(&prog);
  if (low.empty()) {
    set_err("no lowered name for " + name);
    return PBVD_EUNSUPPORTED;
  }
  cudaLibrary_t lib = nullptr;
  cudaKernel_t fn = nullptr;
  cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e == cudaSuccess) e = cudaLibraryGetKernel(&fn, lib, low.c_str());
  if (e != cudaSuccess) {
    set_err(std::string("loading the compiled kernel failed: ") + cudaGetErrorString(e));
    cudaGetLastError();
    if (lib) cudaLibraryUnload(lib);
    return PBVD_ECUDA;
  }
  k.lib[smem] = lib;
  k.fn[smem] = fn;
  return PBVD_OK;
}

JitKernel* get(int jit) {
  if (jit < 0 || jit >= (int)g_jit.size()) return nullptr;
  return g_jit[(size_t)jit];
}

}  // namespace

bool jit_available() { return nvrtc().ok; }

const char* jit_last_error() { return g_jit_err; }

int jit_register(int K, int R, const uint32_t* gens, bool punct, bool var, KernelEntry* out, int cap) {
  if (!jit_available()) return 0;
  std::lock_guard<std::mutex> lk(g_jit_mu);
  const int N = 1 << (K - 1);
  int n = 0;
  // one warp per pair (T = 32) only for codes of 128 states or more (the
  // 64-state codes use their one-warp latency kernel there)
  for (int T = 1; T <= 32 && n < cap; T *= 2) {
    if (T > N / 2 || N / T > 64 || (T == 32 && N < 128)) continue;
    int w = 0, sw = 0;
    shape(K, R, T, &w, &sw);
    if (w <= 0) continue;
    JitKernel* k = new JitKernel();
    k->K = K;
    k->R = R;
    k->T = T;
    for (int r = 0; r < 3; ++r) k->gens[r] = r < R ? gens[r] : 0u;
    k->punct = punct;
    k->var = var;
    g_jit.push_back(k);
    KernelEntry e;
    std::memset(&e, 0, sizeof(e));
    e.K = K;
    e.R = R;
    for (int r = 0; r < 3; ++r) e.gens[r] = k->gens[r];
    e.T = T;
    e.punct = punct;
    e.words_per_stage = w;
    e.scratch_words = sw;
    e.jit = (int)g_jit.size() - 1;
    e.variants = var;
    out[n++] = e;
  }
  return n;
}

int jit_launch(int jit, int smem, const KArgs& a, int grid, int cta, size_t smem_bytes, cudaStream_t s) {
  cudaKernel_t fn = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_jit_mu);
    JitKernel* k = get(jit);
    if (!k) return PBVD_EINVAL;
    if (!k->fn[smem]) {
      const int rc = compile(*k, smem);
      if (rc != PBVD_OK) return rc;
    }
    fn = k->fn[smem];
  }
  KArgs copy = a;
  void* args[] = {&copy};
  const cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(fn), dim3(grid), dim3(cta), args,
                                         smem_bytes, s);
  if (e != cudaSuccess) {
    set_err(std::string("launch: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PBVD_ENOMEM : PBVD_ECUDA;
  }
  return PBVD_OK;
}

bool jit_loaded(int jit, int smem) {
  std::lock_guard<std::mutex> lk(g_jit_mu);
  JitKernel* k = get(jit);
  return k && k->fn[smem] != nullptr;
}

int jit_set_max_smem(int jit, int smem, int bytes) {
  std::lock_guard<std::mutex> lk(g_jit_mu);
  JitKernel* k = get(jit);
  if (!k) return PBVD_EINVAL;
  if (!k->fn[smem]) {
    const int rc = compile(*k, smem);
    if (rc != PBVD_OK) return rc;
  }
  if (bytes <= k->smem_granted[smem]) return PBVD_OK;
  const cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k->fn[smem]),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) {
    set_err(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    return PBVD_ECUDA;
  }
  k->smem_granted[smem] = bytes;
  return PBVD_OK;
}

}  // namespace pbvd
