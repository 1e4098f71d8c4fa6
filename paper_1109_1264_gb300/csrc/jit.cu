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
// interpreter works) where NVRTC is absent; in SALT_JIT_ON mode JIT calls
// then fail with SALT_ERR_CUDA and a message, in SALT_JIT_AUTO mode (the
// default) such programs run on the interpreter.
//
// Compiled kernels are also kept on disk (one file per kernel in the cache
// directory: SALT_JIT_CACHE, else $XDG_CACHE_HOME/salt-jit, else
// $HOME/.cache/salt-jit; salt_jit_cache_dir overrides), keyed by the kernel
// name, the GPU architecture, the NVRTC version and a hash of the embedded
// kernel sources, so a program is compiled once per machine and library
// build.  A file holds a magic word, the FNV-1a hash of its payload, the
// kernel's lowered name and the cubin; a file that fails these checks or
// does not load is ignored and rewritten.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <atomic>
#include <chrono>
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
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
  nvrtcResult (*version)(int*, int*);
};

std::mutex g_mu;
NvrtcApi g_api;
struct Entry {
  cudaLibrary_t lib;
  cudaKernel_t kernel;
};
std::map<std::string, Entry> g_cache;
std::atomic<int32_t> g_mode{SALT_JIT_AUTO};
std::atomic<int64_t> g_compiled{0};
std::atomic<int64_t> g_compile_us{0};
std::atomic<int64_t> g_disk_hits{0};
std::atomic<int64_t> g_disk_writes{0};
thread_local bool t_failed = false;
thread_local bool t_suspended = false;
// the on-disk cache: directory ("" = off), chosen on first use unless set
bool g_dir_set = false;
std::string g_dir;

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Hash of the embedded kernel sources (a rebuilt library with other kernel
// sources must not load the cubins of the old one).
uint64_t sources_hash() {
  static const uint64_t h = [] {
    uint64_t v = 1469598103934665603ull;
    for (int i = 0; i < kJitHeaderCount; ++i) v = fnv1a(kJitHeaderSources[i], strlen(kJitHeaderSources[i]), v);
    return v;
  }();
  return h;
}

// Called with g_mu held.
const std::string& cache_dir() {
  if (g_dir_set) return g_dir;
  g_dir_set = true;
  const char* env = getenv("SALT_JIT_CACHE");
  if (env && (!strcmp(env, "0") || !strcmp(env, "off"))) return g_dir;
  if (env && *env) {
    g_dir = env;
  } else if (const char* x = getenv("XDG_CACHE_HOME"); x && *x) {
    g_dir = std::string(x) + "/salt-jit";
  } else if (const char* hm = getenv("HOME"); hm && *hm) {
    g_dir = std::string(hm) + "/.cache/salt-jit";
  }
  return g_dir;
}

// Creates every missing directory of `dir` (mode 0755); false on failure.
bool make_dirs(const std::string& dir) {
  for (size_t i = 1; i <= dir.size(); ++i) {
    if (i == dir.size() || dir[i] == '/') {
      const std::string part = dir.substr(0, i);
      if (mkdir(part.c_str(), 0755) != 0 && errno != EEXIST) return false;
    }
  }
  return true;
}

constexpr char kMagic[8] = {'S', 'A', 'L', 'T', 'J', 'I', 'T', '1'};

// The cubin and lowered name stored under `path`, if the file is intact.
bool disk_read(const std::string& path, std::string* lowered, std::vector<char>* bin) {
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return false;
  std::vector<char> all;
  char buf[65536];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, f)) > 0) all.insert(all.end(), buf, buf + k);
  fclose(f);
  const size_t head = sizeof kMagic + 8 + 4;
  if (all.size() < head || memcmp(all.data(), kMagic, sizeof kMagic) != 0) return false;
  uint64_t sum;
  uint32_t nlen;
  memcpy(&sum, all.data() + sizeof kMagic, 8);
  memcpy(&nlen, all.data() + sizeof kMagic + 8, 4);
  if (fnv1a(all.data() + head, all.size() - head) != sum || all.size() < head + nlen + 1) return false;
  lowered->assign(all.data() + head, nlen);
  bin->assign(all.begin() + head + nlen, all.end());
  return true;
}

// Writes the file under a temporary name, then renames it into place.
bool disk_write(const std::string& path, const std::string& lowered, const std::vector<char>& bin) {
  std::vector<char> payload(lowered.begin(), lowered.end());
  payload.insert(payload.end(), bin.begin(), bin.end());
  const uint64_t sum = fnv1a(payload.data(), payload.size());
  const uint32_t nlen = (uint32_t)lowered.size();
  const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return false;
  bool ok = fwrite(kMagic, 1, sizeof kMagic, f) == sizeof kMagic && fwrite(&sum, 1, 8, f) == 8 &&
            fwrite(&nlen, 1, 4, f) == 4 && fwrite(payload.data(), 1, payload.size(), f) == payload.size();
  ok = (fclose(f) == 0) && ok;
  if (ok) ok = rename(tmp.c_str(), path.c_str()) == 0;
  if (!ok) unlink(tmp.c_str());
  return ok;
}

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
             sym(h, "nvrtcDestroyProgram", &g_api.destroy) && sym(h, "nvrtcGetErrorString", &g_api.errstr) &&
             sym(h, "nvrtcVersion", &g_api.version);
  if (!g_api.ok) g_api.err = "NVRTC is missing an entry point";
  return g_api;
}

}  // namespace

int32_t jit_mode() { return t_suspended ? SALT_JIT_OFF : g_mode.load(); }
void jit_failure_reset() { t_failed = false; }
bool jit_failed() { return t_failed; }
void jit_suspend(bool on) { t_suspended = on; }

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
  t_failed = true;  // cleared below once a kernel is in hand
  NvrtcApi& a = api();
  if (!a.ok) return report_error(SALT_ERR_CUDA, a.err);
  const auto t0 = std::chrono::steady_clock::now();
  const std::string arch = "-arch=sm_" + std::to_string(major * 10 + minor) + "a";
  int nv_major = 0, nv_minor = 0;
  a.version(&nv_major, &nv_minor);
  const std::string tag = name + "|" + arch + "|nvrtc " + std::to_string(nv_major) + "." + std::to_string(nv_minor);
  char fname[64];
  snprintf(fname, sizeof fname, "/%016llx-%016llx.cubin", (unsigned long long)fnv1a(tag.data(), tag.size()),
           (unsigned long long)sources_hash());
  const std::string dir = cache_dir();
  const std::string path = dir.empty() ? std::string() : dir + fname;
  std::string lowered_name;
  std::vector<char> bin;
  Entry e{};
  bool from_disk = false;
  if (!path.empty() && disk_read(path, &lowered_name, &bin)) {
    cudaError_t ce = cudaLibraryLoadData(&e.lib, bin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&e.kernel, e.lib, lowered_name.c_str());
    if (ce == cudaSuccess) {
      from_disk = true;
    } else {
      cudaGetLastError();  // a stale or foreign file: compile afresh below
      if (e.lib) cudaLibraryUnload(e.lib);
      e = Entry{};
    }
  }
  if (!from_disk) {
    nvrtcProgram prog = nullptr;
    nvrtcResult r = a.create(&prog, "#include \"fused.cuh\"\n", "salt_jit.cu", kJitHeaderCount, kJitHeaderSources,
                             kJitHeaderNames);
    if (r != NVRTC_SUCCESS) return report_error(SALT_ERR_CUDA, std::string("nvrtcCreateProgram: ") + a.errstr(r));
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
    lowered_name = lowered ? lowered : "";
    size_t nbin = 0;
    a.cubin_size(prog, &nbin);
    bin.assign(nbin, 0);
    if (nbin) a.cubin(prog, bin.data());
    a.destroy(&prog);
    if (lowered_name.empty() || nbin == 0) return report_error(SALT_ERR_CUDA, "NVRTC produced no kernel");
    cudaError_t ce = cudaLibraryLoadData(&e.lib, bin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&e.kernel, e.lib, lowered_name.c_str());
    if (ce != cudaSuccess)
      return report_error(SALT_ERR_CUDA, std::string("loading the JIT kernel: ") + cudaGetErrorString(ce));
    if (!path.empty() && make_dirs(dir) && disk_write(path, lowered_name, bin)) g_disk_writes.fetch_add(1);
    g_compiled.fetch_add(1);
    g_compile_us.fetch_add(
        std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count());
  } else {
    g_disk_hits.fetch_add(1);
  }
  g_cache[key] = e;
  t_failed = false;
  *kernel_out = (const void*)e.kernel;
  return SALT_OK;
}

}  // namespace salt

extern "C" {

salt_status salt_set_jit(int32_t mode) {
  if (mode != SALT_JIT_OFF && mode != SALT_JIT_ON && mode != SALT_JIT_AUTO)
    return salt::report_error(SALT_ERR_ARG, "mode must be SALT_JIT_OFF, SALT_JIT_ON or SALT_JIT_AUTO");
  salt::g_mode.store(mode);
  return SALT_OK;
}

salt_status salt_jit_cache_dir(const char* dir) {
  std::lock_guard<std::mutex> lk(salt::g_mu);
  salt::g_dir_set = true;
  salt::g_dir = dir ? dir : "";
  return SALT_OK;
}

salt_status salt_jit_cache_stats(int64_t* disk_hits, int64_t* disk_writes, char* dir, int32_t dir_len) {
  if (disk_hits) *disk_hits = salt::g_disk_hits.load();
  if (disk_writes) *disk_writes = salt::g_disk_writes.load();
  if (dir && dir_len > 0) {
    std::lock_guard<std::mutex> lk(salt::g_mu);
    const std::string& d = salt::cache_dir();
    snprintf(dir, (size_t)dir_len, "%s", d.c_str());
  }
  return SALT_OK;
}

salt_status salt_jit_stats(int32_t* mode, int64_t* kernels, double* compile_ms) {
  if (mode) *mode = salt::g_mode.load();
  if (kernels) *kernels = salt::g_compiled.load();
  if (compile_ms) *compile_ms = salt::g_compile_us.load() / 1000.0;
  return SALT_OK;
}

}  // extern "C"
