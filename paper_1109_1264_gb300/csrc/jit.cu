// Run-time instantiation of the fused kernel for programs that have no
// compile-time instantiation.
//
// The paper builds the loop for each expression at compile time (Section 2:
// expression templates are code generation at compile time).  A library that
// receives programs at run time can do the same one step later: the canonical
// program is spelled out as the template argument list of fused_kernel (the
// very template the compiled shapes use, from fused.cuh), NVRTC compiles that
// instantiation for the current GPU, and the cubin is loaded and cached per
// (device, program, dtype, unroll, vector width).  The result is the fused
// one-pass kernel -- same per-element operations, so the same bits as the
// interpreter and the oracle -- instead of the interpreter.
//
// NVRTC is opened with dlopen on first use, so the library loads (and the
// interpreter works) where NVRTC is absent; JIT calls then fail with
// SALT_ERR_CUDA and a message.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/salt.h"
#include "host.h"
#include "internal.h"
#include "jit_sources.inc"  // generated by build.py: the device headers as strings

namespace salt {
namespace {

struct NvrtcApi {
  bool tried = false, ok = false;
  std::string err;
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
  nvrtcResult (*add_name)(nvrtcProgram, const char*);
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*);
  nvrtcResult (*lowered)(nvrtcProgram, const char*, const char**);
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*);
  nvrtcResult (*cubin)(nvrtcProgram, char*);
  nvrtcResult (*log_size)(nvrtcProgram, size_t*);
  nvrtcResult (*log)(nvrtcProgram, char*);
  nvrtcResult (*destroy)(nvrtcProgram*);
  const char* (*errstr)(nvrtcResult);
};

std::mutex g_mu;
NvrtcApi g_api;
struct Entry {
  cudaLibrary_t lib;
  cudaKernel_t kernel;
};
std::map<std::string, Entry> g_cache;
std::atomic<int32_t> g_mode{SALT_JIT_OFF};
std::atomic<int64_t> g_compiled{0};
std::atomic<int64_t> g_compile_us{0};

template <typename F>
bool sym(void* h, const char* name, F* out) {
  *out = reinterpret_cast<F>(dlsym(h, name));
  return *out != nullptr;
}

// Called with g_mu held.
NvrtcApi& api() {
  if (g_api.tried) return g_api;
  g_api.tried = true;
  void* h = nullptr;
  for (const char* name : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so"}) {
    h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
    if (h) break;
  }
  if (!h) {
    g_api.err = "NVRTC (libnvrtc.so) could not be loaded";
    return g_api;
  }
  g_api.ok = sym(h, "nvrtcCreateProgram", &g_api.create) && sym(h, "nvrtcAddNameExpression", &g_api.add_name) &&
             sym(h, "nvrtcCompileProgram", &g_api.compile) && sym(h, "nvrtcGetLoweredName", &g_api.lowered) &&
             sym(h, "nvrtcGetCUBINSize", &g_api.cubin_size) && sym(h, "nvrtcGetCUBIN", &g_api.cubin) &&
             sym(h, "nvrtcGetProgramLogSize", &g_api.log_size) && sym(h, "nvrtcGetProgramLog", &g_api.log) &&
             sym(h, "nvrtcDestroyProgram", &g_api.destroy) && sym(h, "nvrtcGetErrorString", &g_api.errstr);
  if (!g_api.ok) g_api.err = "NVRTC is missing an entry point";
  return g_api;
}

}  // namespace

int32_t jit_mode() { return g_mode.load(); }

salt_status jit_kernel(const Canonical& c, int is_f32, int unroll, int vec_bytes, bool ds,
                       const void** kernel_out) {
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  // vec_bytes == 0: the element-access kernel (unaligned or strided operands)
  std::string name = vec_bytes ? "salt::fused_kernel<salt::Prog<" : "salt::strided_kernel<salt::Prog<";
  for (int i = 0; i < c.len; ++i) name += (i ? "," : "") + std::to_string(c.code[i]);
  name += ">," + std::string(is_f32 ? "float" : "double") + "," + std::to_string(unroll);
  name += vec_bytes ? "," + std::to_string(vec_bytes) + (ds ? ",true>" : ">") : ">";
  const std::string key = std::to_string(dev) + "|" + name;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(key);
  if (it != g_cache.end()) {
    *kernel_out = (const void*)it->second.kernel;
    return SALT_OK;
  }
  NvrtcApi& a = api();
  if (!a.ok) return report_error(SALT_ERR_CUDA, a.err);
  const auto t0 = std::chrono::steady_clock::now();
  nvrtcProgram prog = nullptr;
  nvrtcResult r = a.create(&prog, "#include \"fused.cuh\"\n", "salt_jit.cu", kJitHeaderCount, kJitHeaderSources,
                           kJitHeaderNames);
  if (r != NVRTC_SUCCESS) return report_error(SALT_ERR_CUDA, std::string("nvrtcCreateProgram: ") + a.errstr(r));
  const std::string arch = "-arch=sm_" + std::to_string(major * 10 + minor) + "a";
  const char* opts[] = {arch.c_str(), "-std=c++17", "--fmad=false"};
  r = a.add_name(prog, name.c_str());
  if (r == NVRTC_SUCCESS) r = a.compile(prog, 3, opts);
  if (r != NVRTC_SUCCESS) {
    size_t n = 0;
    a.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) a.log(prog, &log[0]);
    a.destroy(&prog);
    return report_error(SALT_ERR_CUDA, std::string("NVRTC compile failed: ") + a.errstr(r) + "\n" + log);
  }
  const char* lowered = nullptr;
  a.lowered(prog, name.c_str(), &lowered);
  const std::string lowered_name = lowered ? lowered : "";
  size_t nbin = 0;
  a.cubin_size(prog, &nbin);
  std::vector<char> bin(nbin);
  if (nbin) a.cubin(prog, bin.data());
  a.destroy(&prog);
  if (lowered_name.empty() || nbin == 0) return report_error(SALT_ERR_CUDA, "NVRTC produced no kernel");
  Entry e{};
  cudaError_t ce = cudaLibraryLoadData(&e.lib, bin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&e.kernel, e.lib, lowered_name.c_str());
  if (ce != cudaSuccess) return report_error(SALT_ERR_CUDA, std::string("loading the JIT kernel: ") + cudaGetErrorString(ce));
  g_cache[key] = e;
  g_compiled.fetch_add(1);
  g_compile_us.fetch_add(
      std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count());
  *kernel_out = (const void*)e.kernel;
  return SALT_OK;
}

}  // namespace salt

extern "C" {

salt_status salt_set_jit(int32_t mode) {
  if (mode != SALT_JIT_OFF && mode != SALT_JIT_ON) return salt::report_error(SALT_ERR_ARG, "mode must be 0 or 1");
  salt::g_mode.store(mode);
  return SALT_OK;
}

salt_status salt_jit_stats(int32_t* mode, int64_t* kernels, double* compile_ms) {
  if (mode) *mode = salt::g_mode.load();
  if (kernels) *kernels = salt::g_compiled.load();
  if (compile_ms) *compile_ms = salt::g_compile_us.load() / 1000.0;
  return SALT_OK;
}

}  // extern "C"
