// Rule-specialised asynchronous kernel: source generation, NVRTC compile,
// loading and caches (see inet_jit.h).
#include "inet_jit.h"

#include "inet.h"

#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

// kJitHeaderNames / kJitHeaderTexts / kJitHeaderCount: the device headers,
// embedded by the build (lib/inet_jit_src.inc), so that the library compiles
// the same sources it was built from wherever it runs.
#include "inet_jit_src.inc"

namespace inet {
namespace {

// Minimal standard headers for NVRTC, which has no host include tree: the
// device headers only need the fixed-width integer types and size_t.
const char* const kShimNames[] = {"cstdint", "stdint.h", "stddef.h", "cuda_runtime.h"};
const char* const kShimTexts[] = {
    "#pragma once\n"
    "typedef signed char int8_t; typedef unsigned char uint8_t;\n"
    "typedef short int16_t; typedef unsigned short uint16_t;\n"
    "typedef int int32_t; typedef unsigned int uint32_t;\n"
    "typedef long long int64_t; typedef unsigned long long uint64_t;\n",
    "#pragma once\n#include <cstdint>\n",
    "#pragma once\ntypedef unsigned long size_t;\n",
    "#pragma once\n",
};

uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; i++) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

// NVRTC entry points, resolved once with dlopen.
struct Nvrtc {
  bool ok = false;
  std::string why;
  int major = 0, minor = 0;
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*) = nullptr;
  nvrtcResult (*add_name)(nvrtcProgram, const char*) = nullptr;
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*) = nullptr;
  nvrtcResult (*log_size)(nvrtcProgram, size_t*) = nullptr;
  nvrtcResult (*log)(nvrtcProgram, char*) = nullptr;
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*) = nullptr;
  nvrtcResult (*cubin)(nvrtcProgram, char*) = nullptr;
  nvrtcResult (*lowered)(nvrtcProgram, const char*, const char**) = nullptr;
  nvrtcResult (*destroy)(nvrtcProgram*) = nullptr;
  nvrtcResult (*version)(int*, int*) = nullptr;
};

const Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    // $INET_NVRTC_LIB names the library to use, and only it; otherwise the
    // loader's search path, then the CUDA installation
    std::vector<std::string> cands;
    if (const char* e = getenv("INET_NVRTC_LIB")) {
      cands.push_back(e);
    } else {
      cands.push_back("libnvrtc.so.13");
      cands.push_back("libnvrtc.so");
      const char* homes[] = {getenv("CUDA_HOME"), getenv("CUDA_PATH"), "/usr/local/cuda"};
      for (const char* home : homes) {
        if (!home) continue;
        cands.push_back(std::string(home) + "/lib64/libnvrtc.so.13");
        cands.push_back(std::string(home) + "/lib64/libnvrtc.so");
      }
    }
    void* h = nullptr;
    for (const std::string& c : cands)
      if ((h = dlopen(c.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) {
      n.why = "NVRTC library not found (libnvrtc.so.13)";
      return;
    }
    bool all = true;
    auto sym = [&](auto& fp, const char* name) {
      fp = reinterpret_cast<std::remove_reference_t<decltype(fp)>>(dlsym(h, name));
      if (!fp) all = false;
    };
    sym(n.create, "nvrtcCreateProgram");
    sym(n.add_name, "nvrtcAddNameExpression");
    sym(n.compile, "nvrtcCompileProgram");
    sym(n.log_size, "nvrtcGetProgramLogSize");
    sym(n.log, "nvrtcGetProgramLog");
    sym(n.cubin_size, "nvrtcGetCUBINSize");
    sym(n.cubin, "nvrtcGetCUBIN");
    sym(n.lowered, "nvrtcGetLoweredName");
    sym(n.destroy, "nvrtcDestroyProgram");
    sym(n.version, "nvrtcVersion");
    if (!all) {
      n.why = "NVRTC library lacks an entry point";
      return;
    }
    n.version(&n.major, &n.minor);
    n.ok = true;
  });
  return n;
}

// Directory of the on-disk cache: $INET_JIT_CACHE ("" turns it off), else
// jit-cache beside this library.
std::string cache_dir() {
  if (const char* e = getenv("INET_JIT_CACHE")) return e;
  Dl_info info;
  if (dladdr(reinterpret_cast<void*>(&rules_key), &info) && info.dli_fname) {
    std::string p = info.dli_fname;
    const size_t s = p.rfind('/');
    return (s == std::string::npos ? std::string(".") : p.substr(0, s)) + "/jit-cache";
  }
  return "";
}

// A cache file: a line with the kernel's lowered name, then the cubin.
bool read_cached(const std::string& path, std::string* name, std::vector<char>* cubin) {
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return false;
  std::vector<char> all;
  char buf[1 << 16];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, f)) > 0) all.insert(all.end(), buf, buf + k);
  fclose(f);
  const char magic[] = "INETJIT1 ";
  const size_t ml = sizeof magic - 1;
  if (all.size() < ml || memcmp(all.data(), magic, ml) != 0) return false;
  size_t nl = ml;
  while (nl < all.size() && all[nl] != '\n') nl++;
  if (nl >= all.size() || nl + 1 == all.size()) return false;
  name->assign(all.data() + ml, nl - ml);
  cubin->assign(all.begin() + (long)nl + 1, all.end());
  return true;
}

void write_cached(const std::string& dir, const std::string& path, const std::string& name,
                  const std::vector<char>& cubin) {
  if (dir.empty()) return;
  mkdir(dir.c_str(), 0755);
  const std::string tmp = path + ".tmp" + std::to_string((unsigned long)getpid());
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return;
  bool ok = fprintf(f, "INETJIT1 %s\n", name.c_str()) > 0 && fwrite(cubin.data(), 1, cubin.size(), f) == cubin.size();
  ok = (fclose(f) == 0) && ok;
  if (!ok || rename(tmp.c_str(), path.c_str()) != 0) remove(tmp.c_str());
}

struct Loaded {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
};

std::mutex g_mu;
std::map<std::string, Loaded> g_loaded;  // by cache key: kept for the life of the process

}  // namespace

uint64_t rules_key(const Template* t, size_t n) {
  const uint64_t h = fnv1a(&n, sizeof n);
  return n ? fnv1a(t, n * sizeof(Template), h) : h;
}

std::string jit_source(const Template* t, size_t n) {
  std::string s;
  char buf[96];
  s += "// generated: k_async specialised for one rule set\n#include \"inet_async.cuh\"\nnamespace inet {\n";
  s += "struct JitRules {\n";
  snprintf(buf, sizeof buf, "  static constexpr int kN = %zu;\n", n);
  s += buf;
  snprintf(buf, sizeof buf, "  static constexpr unsigned long long kKey = %lluull;\n", (unsigned long long)rules_key(t, n));
  s += buf;
  s += "  static constexpr Template kT[kN] = {\n";
  for (size_t i = 0; i < n; i++) {
    const Template& r = t[i];
    snprintf(buf, sizeof buf, "    {%u, %u, %u, %u, {", r.n_new, r.n_fresh, r.n_link, r.rule);
    s += buf;
    for (int j = 0; j < kMaxNew; j++) s += std::to_string(r.lab[j]) + (j + 1 < kMaxNew ? ", " : "}, {");
    for (int j = 0; j < kMaxNew; j++) {
      snprintf(buf, sizeof buf, "{%u, %u, %u}%s", r.src[j][0], r.src[j][1], r.src[j][2], j + 1 < kMaxNew ? ", " : "}, {");
      s += buf;
    }
    for (int k = 0; k < kMaxLink; k++) {
      snprintf(buf, sizeof buf, "{%u, %u}%s", r.link[k][0], r.link[k][1], k + 1 < kMaxLink ? ", " : "}, ");
      s += buf;
    }
    snprintf(buf, sizeof buf, "{%u, %u}, {0}},\n", r.lhs[0], r.lhs[1]);
    s += buf;
  }
  s += "  };\n};\n}  // namespace inet\n";
  return s;
}

bool jit_async(const Template* t, size_t n, bool track, const std::string& arch, bool load, JitResult* out,
               std::string* err) {
  *out = JitResult{};
  if (n == 0 || n > (size_t)INET_MAX_RULES) {
    *err = "no rules to specialise for";
    return false;
  }
  const Nvrtc& nv = nvrtc();
  const std::string src = jit_source(t, n);
  const std::string expr = std::string("inet::k_async<") + (track ? "true" : "false") + ", inet::JitRules>";
  const std::string arch_opt = "--gpu-architecture=" + arch;
  const char* const opts[] = {arch_opt.c_str(), "-std=c++17", "-default-device", "-lineinfo",
                              "--diag-suppress=177,186", "-DINET_JIT=1"};
  const int n_opts = (int)(sizeof opts / sizeof opts[0]);
  // the key: everything the cubin depends on
  uint64_t h = fnv1a(src.data(), src.size());
  for (int i = 0; i < kJitHeaderCount; i++) h = fnv1a(kJitHeaderTexts[i], strlen(kJitHeaderTexts[i]), h);
  for (int i = 0; i < n_opts; i++) h = fnv1a(opts[i], strlen(opts[i]), h);
  h = fnv1a(&nv.major, sizeof nv.major, h);
  h = fnv1a(&nv.minor, sizeof nv.minor, h);
  char keybuf[64];
  snprintf(keybuf, sizeof keybuf, "k_async_%s_%d_%016llx", arch.c_str(), track ? 1 : 0, (unsigned long long)h);
  const std::string key = keybuf;

  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_loaded.find(key);
  if (it != g_loaded.end() && (!load || it->second.kern)) {
    out->fn = load ? reinterpret_cast<const void*>(it->second.kern) : nullptr;
    out->from_memory = true;
    return true;
  }
  const std::string dir = cache_dir();
  const std::string path = dir.empty() ? std::string() : dir + "/" + key + ".cubin";
  std::string name;
  std::vector<char> cubin;
  // NVRTC: the cubin of the generated source, written to the disk cache
  auto compile = [&]() -> bool {
    if (!nv.ok) {
      *err = nv.why;
      return false;
    }
    std::vector<const char*> hn, ht;
    for (int i = 0; i < 4; i++) {
      hn.push_back(kShimNames[i]);
      ht.push_back(kShimTexts[i]);
    }
    for (int i = 0; i < kJitHeaderCount; i++) {
      hn.push_back(kJitHeaderNames[i]);
      ht.push_back(kJitHeaderTexts[i]);
    }
    nvrtcProgram prog = nullptr;
    if (nv.create(&prog, src.c_str(), "inet_jit.cu", (int)hn.size(), ht.data(), hn.data()) != NVRTC_SUCCESS) {
      *err = "nvrtcCreateProgram failed";
      return false;
    }
    bool ok = nv.add_name(prog, expr.c_str()) == NVRTC_SUCCESS;
    const auto t0 = std::chrono::steady_clock::now();
    ok = ok && nv.compile(prog, n_opts, opts) == NVRTC_SUCCESS;
    out->compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (!ok) {
      size_t ls = 0;
      std::string log;
      if (nv.log_size(prog, &ls) == NVRTC_SUCCESS && ls > 1) {
        log.resize(ls);
        nv.log(prog, &log[0]);
      }
      nv.destroy(&prog);
      *err = "NVRTC compile failed: " + log.substr(0, 2000);
      return false;
    }
    const char* low = nullptr;
    size_t cs = 0;
    ok = nv.lowered(prog, expr.c_str(), &low) == NVRTC_SUCCESS && low && nv.cubin_size(prog, &cs) == NVRTC_SUCCESS;
    if (ok) {
      name = low;
      cubin.resize(cs);
      ok = nv.cubin(prog, cubin.data()) == NVRTC_SUCCESS;
    }
    nv.destroy(&prog);
    if (!ok) {
      *err = "NVRTC produced no cubin";
      return false;
    }
    if (!path.empty()) write_cached(dir, path, name, cubin);
    return true;
  };
  if (!path.empty() && read_cached(path, &name, &cubin)) {
    out->from_disk = true;
  } else if (!compile()) {
    return false;
  }
  Loaded L;
  if (load) {
    // the image is checked when it is loaded or, with lazy loading, when the
    // kernel is looked up
    auto load_kernel = [&]() -> cudaError_t {
      L = Loaded{};
      cudaError_t e = cudaLibraryLoadData(&L.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
      if (e == cudaSuccess) e = cudaLibraryGetKernel(&L.kern, L.lib, name.c_str());
      if (e != cudaSuccess) {
        if (L.lib) cudaLibraryUnload(L.lib);
        L = Loaded{};
        cudaGetLastError();  // the failure is reported here, not to the context's next call
      }
      return e;
    };
    cudaError_t e = load_kernel();
    if (e != cudaSuccess && out->from_disk) {
      // a damaged cache file: compile again and replace it
      out->from_disk = false;
      remove(path.c_str());
      if (!compile()) return false;
      e = load_kernel();
    }
    if (e != cudaSuccess) {
      *err = std::string("loading the specialised kernel failed: ") + cudaGetErrorString(e);
      return false;
    }
    out->fn = reinterpret_cast<const void*>(L.kern);
  }
  g_loaded[key] = L;
  return true;
}

}  // namespace inet
