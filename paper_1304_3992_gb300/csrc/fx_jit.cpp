// fx_jit.cpp -- the streaming first pass compiled at run time for one
// parameter set (fx_specialize).
//
// A packed FP32x2 operand that comes from the kernel parameters needs a
// register pair holding the value twice; under the kernel's register cap the
// twelve LoG ring weights and the two contrast thresholds then cost register
// moves and spills.  fx_specialize compiles fx::stream_kernel (fx_stream.cuh)
// with NVRTC, the weights and thresholds of one parameter set being
// compile-time constants (instruction immediates), and caches the kernel per
// device, pixel size, load path, strip class and constants; it does the same
// for the batched path's group kernel (fx::batch_kernel_fast), each for both
// load paths.  fx_extract and the host-buffer path launch them whenever their
// parameters match, and plans created afterwards put them in their graphs; the
// arithmetic is the same, so the masks are identical either way.  NVRTC is
// loaded on first use (dlopen); without it fx_specialize reports
// FX_ERR_UNSUPPORTED and every call runs the precompiled kernels.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fx_internal.h"

#ifndef FX_SRC_DIR
#define FX_SRC_DIR "."
#endif
#ifndef FX_INC_DIR
#define FX_INC_DIR "."
#endif
#ifndef FX_CUDA_LIB_DIR
#define FX_CUDA_LIB_DIR "/usr/local/cuda/lib64"
#endif

namespace fx {
namespace {

struct Nvrtc {
  bool ok = false;
  nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *, const char *const *);
  nvrtcResult (*add_name)(nvrtcProgram, const char *);
  nvrtcResult (*compile)(nvrtcProgram, int, const char *const *);
  nvrtcResult (*log_size)(nvrtcProgram, size_t *);
  nvrtcResult (*log)(nvrtcProgram, char *);
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t *);
  nvrtcResult (*cubin)(nvrtcProgram, char *);
  nvrtcResult (*lowered)(nvrtcProgram, const char *, const char **);
  nvrtcResult (*destroy)(nvrtcProgram *);
};

template <typename F>
bool sym(void *h, const char *name, F *out) {
  *out = reinterpret_cast<F>(dlsym(h, name));
  return *out != nullptr;
}

const Nvrtc &nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char *names[] = {FX_CUDA_LIB_DIR "/libnvrtc.so.13", "libnvrtc.so.13", FX_CUDA_LIB_DIR "/libnvrtc.so",
                           "libnvrtc.so"};
    void *h = nullptr;
    for (const char *nm : names)
      if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) return;
    n.ok = sym(h, "nvrtcCreateProgram", &n.create) && sym(h, "nvrtcAddNameExpression", &n.add_name) &&
           sym(h, "nvrtcCompileProgram", &n.compile) && sym(h, "nvrtcGetProgramLogSize", &n.log_size) &&
           sym(h, "nvrtcGetProgramLog", &n.log) && sym(h, "nvrtcGetCUBINSize", &n.cubin_size) &&
           sym(h, "nvrtcGetCUBIN", &n.cubin) && sym(h, "nvrtcGetLoweredName", &n.lowered) &&
           sym(h, "nvrtcDestroyProgram", &n.destroy);
  });
  return n;
}

// The kernel variant and the constants it bakes in.
struct Variant {
  int kind;  // 0: fx_extract's first pass (stream_kernel), 1: the batched group kernel (batch_kernel_fast)
  int device, elem, pair, rm_class, f32log, sd2, src_z, nhmf, hmf[FX_MAX_HMF_LEVELS], check;
  float w[2][6], ntzc[2];
};

Variant variant_of(int kind, int device, const KParams &kp, int elem, bool pair, int rm_class) {
  Variant v;
  std::memset(&v, 0, sizeof v);
  v.kind = kind;
  v.device = device;
  v.elem = elem;
  v.pair = pair ? 1 : 0;
  v.rm_class = rm_class;
  v.f32log = kp.f32log ? 1 : 0;
  v.src_z = kp.source == 1 ? 1 : 0;
  v.sd2 = (!v.src_z && !kp.sd_same) ? 1 : 0;
  v.nhmf = kp.nhmf;
  for (int l = 0; l < kp.nhmf && l < FX_MAX_HMF_LEVELS; ++l) v.hmf[l] = kp.hmf[l];
  // the first pass's bound check (the kernels' A::kChecked holds for every FP32 first pass)
  v.check = kp.fbound < (elem == 1 ? 255 : 65535) ? 1 : 0;
  std::memcpy(v.w, kp.ringf, sizeof v.w);
  std::memcpy(v.ntzc, kp.ntzc1f, sizeof v.ntzc);
  return v;
}

std::string key_of(const Variant &v) { return std::string(reinterpret_cast<const char *>(&v), sizeof v); }

std::mutex g_mu;
std::map<std::string, const void *> g_cache;
int g_entries = 0;  // read without the lock: 0 means no call can hit

std::string hexf(float x) {
  char b[48];
  std::snprintf(b, sizeof b, "%af", static_cast<double>(x));
  return b;
}

std::string name_of(const Variant &v) {
  return std::string(v.kind ? "fx::batch_kernel_fast<" : "fx::stream_kernel<") + (v.elem == 1 ? "unsigned char" : "unsigned short") + ", " +
         (v.f32log ? "true" : "false") + ", " + (v.pair ? "true" : "false") + ", " + (v.sd2 ? "true" : "false") +
         ", " + (v.src_z ? "true" : "false") + ", " + std::to_string(v.rm_class) + ", JitConsts>";
}

std::string source_of(const Variant &v) {
  std::string s =
      "typedef signed char int8_t; typedef unsigned char uint8_t; typedef short int16_t;\n"
      "typedef unsigned short uint16_t; typedef int int32_t; typedef unsigned int uint32_t;\n"
      "typedef long long int64_t; typedef unsigned long long uint64_t; typedef unsigned long uintptr_t;\n"
      "typedef unsigned long size_t;\n"
      "#include \"fx_stream.cuh\"\n#include \"fx_plan_kernels.cuh\"\n"
      "struct JitConsts {\n"
      "  static constexpr bool kStatic = true;\n"
      "  static __device__ __forceinline__ float w(int f, int c) {\n"
      "    constexpr float t[2][6] = {";
  for (int f = 0; f < 2; ++f) {
    s += f ? ", {" : "{";
    for (int c = 0; c < 6; ++c) s += (c ? ", " : "") + hexf(v.w[f][c]);
    s += "}";
  }
  s += "};\n    return t[f][c];\n  }\n";
  s += "  static __device__ __forceinline__ float ntzc(int f) { return f ? " + hexf(v.ntzc[1]) + " : " +
       hexf(v.ntzc[0]) + "; }\n";
  s += "  static constexpr int kNhmf = " + std::to_string(v.nhmf) + ";\n";
  s += "  static constexpr bool kCheck = " + std::string(v.check ? "true" : "false") + ";\n";
  s += "  static __device__ __forceinline__ int hmf(int l) { constexpr int t[" + std::to_string(FX_MAX_HMF_LEVELS) +
       "] = {";
  for (int l = 0; l < FX_MAX_HMF_LEVELS; ++l) s += (l ? ", " : "") + std::to_string(v.hmf[l]);
  s += "}; return t[l]; }\n};\n";
  return s;
}

// Compiles and loads one variant; nullptr (and a message on stderr) on failure.
const void *build(const Variant &v) {
  const Nvrtc &n = nvrtc();
  if (!n.ok) return nullptr;
  const std::string src = source_of(v), name = "&" + name_of(v);
  nvrtcProgram prog;
  if (n.create(&prog, src.c_str(), "fx_specialized.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) return nullptr;
  const void *kernel = nullptr;
  // -default-device: the headers' unannotated functions (the C ABI declarations,
  // constexpr helpers) are taken as device functions
  std::vector<std::string> opts = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device",
                                   std::string("-I") + FX_SRC_DIR, std::string("-I") + FX_INC_DIR};
#ifdef FX_WARPS_PER_CTA
  opts.push_back("-DFX_WARPS_PER_CTA=" + std::to_string(FX_WARPS_PER_CTA));
#endif
#ifdef FX_FIRST_PASS_CTAS
  opts.push_back("-DFX_FIRST_PASS_CTAS=" + std::to_string(FX_FIRST_PASS_CTAS));
#endif
#ifdef FX_BATCH_CTAS
  opts.push_back("-DFX_BATCH_CTAS=" + std::to_string(FX_BATCH_CTAS));
#endif
  std::vector<const char *> argv;
  for (const auto &o : opts) argv.push_back(o.c_str());
  n.add_name(prog, name.c_str());
  if (n.compile(prog, static_cast<int>(argv.size()), argv.data()) == NVRTC_SUCCESS) {
    size_t sz = 0;
    const char *lowered = nullptr;
    if (n.cubin_size(prog, &sz) == NVRTC_SUCCESS && sz > 0 && n.lowered(prog, name.c_str(), &lowered) == NVRTC_SUCCESS) {
      std::vector<char> cubin(sz);
      cudaLibrary_t lib;
      cudaKernel_t k;
      if (n.cubin(prog, cubin.data()) == NVRTC_SUCCESS &&
          cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) == cudaSuccess &&
          cudaLibraryGetKernel(&k, lib, lowered) == cudaSuccess)
        kernel = reinterpret_cast<const void *>(k);
    }
  } else {
    size_t ls = 0;
    if (n.log_size(prog, &ls) == NVRTC_SUCCESS && ls > 1) {
      std::vector<char> log(ls);
      if (n.log(prog, log.data()) == NVRTC_SUCCESS) std::fprintf(stderr, "fx_specialize: %s\n", log.data());
    }
  }
  n.destroy(&prog);
  return kernel;
}

}  // namespace

namespace {
const void *lookup(int kind, const KParams &kp, int elem, bool pair, int rm_class) {
  if (__atomic_load_n(&g_entries, __ATOMIC_ACQUIRE) == 0) return nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  const std::string key = key_of(variant_of(kind, dev, kp, elem, pair, rm_class));
  std::lock_guard<std::mutex> lock(g_mu);
  const auto it = g_cache.find(key);
  return it == g_cache.end() ? nullptr : it->second;
}
}  // namespace

const void *specialized_kernel(const KParams &kp, int elem, bool pair, int rm_class) {
  return lookup(0, kp, elem, pair, rm_class);
}
const void *specialized_batch_kernel(const KParams &kp, int elem, bool pair, int rm_class) {
  return lookup(1, kp, elem, pair, rm_class);
}

// Compiles the first pass of fx_extract and the batched group kernel for kp,
// each for both load paths (aligned words, and rows that are not 4-byte
// aligned), on the current device; the four compiles run in parallel.
fx_status specialize(const KParams &kp, int elem) {
  if (checked_build()) return FX_ERR_UNSUPPORTED;  // its kernels count range-check failures
  if (kp.fbound < 0 || !fast_path_supported(kp)) return FX_ERR_UNSUPPORTED;
  if (!nvrtc().ok) return FX_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FX_ERR_CUDA;
  std::vector<Variant> todo;
  for (int kind = 0; kind < 2; ++kind)
    for (int pair = 1; pair >= 0; --pair) {
      const Variant v = variant_of(kind, dev, kp, elem, pair != 0, strip_class(kp));
      std::lock_guard<std::mutex> lock(g_mu);
      if (!g_cache.count(key_of(v))) todo.push_back(v);
    }
  std::vector<const void *> built(todo.size(), nullptr);
  std::vector<std::thread> threads;
  for (size_t i = 0; i < todo.size(); ++i)
    threads.emplace_back([&, i] {
      // each thread loads its cubin on the caller's device
      if (cudaSetDevice(dev) == cudaSuccess) built[i] = build(todo[i]);
    });
  for (auto &t : threads) t.join();
  std::lock_guard<std::mutex> lock(g_mu);
  bool all = true;
  for (size_t i = 0; i < todo.size(); ++i) {
    if (built[i]) g_cache[key_of(todo[i])] = built[i];
    else all = false;
  }
  __atomic_store_n(&g_entries, static_cast<int>(g_cache.size()), __ATOMIC_RELEASE);
  return all ? FX_OK : FX_ERR_UNSUPPORTED;
}

}  // namespace fx

extern "C" fx_status fx_specialize(const fx_params *params, fx_dtype dtype) {
  if (!params || params->struct_size != sizeof(fx_params) || (dtype != FX_U8 && dtype != FX_U16))
    return FX_ERR_INVALID_ARG;
  fx::KParams kp;
  const fx_status st = fx::make_kparams(params, dtype == FX_U8 ? 255 : 65535, &kp);
  if (st != FX_OK) return st;
  return fx::specialize(kp, dtype == FX_U8 ? 1 : 2);
}
