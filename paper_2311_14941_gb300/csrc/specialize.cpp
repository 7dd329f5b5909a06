// specialize.cpp -- run-time compilation of the mechanism-specialised integration kernels (specialize.h).
//
// NVRTC is opened with dlopen, so the library does not depend on it unless specialisation is asked for.
// The device headers are embedded at build time (rtc_headers.inc, written by build.py from the same files
// the library's own kernels are compiled from).  Compiled cubins are kept in a cache directory
// (CHEM_RTC_CACHE, else rtc_cache beside the library), keyed by a hash of the source, the headers, the
// options and the compiler's version.
#include "specialize.h"

#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <thread>
#include <vector>

#include "rtc_headers.inc"   // kRtcHeaderNames, kRtcHeaderTexts, kRtcHeaderCount

namespace chemgb {
namespace {

struct Nvrtc {
  decltype(&nvrtcVersion) version = nullptr;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcAddNameExpression) add_name = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetLoweredName) lowered = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&nvrtcGetErrorString) error_string = nullptr;
  bool ok = false;
  std::string why;
};

const Nvrtc& nvrtc() {
  static Nvrtc api;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void* lib = nullptr;
    for (const char* n : names)
      if ((lib = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!lib) {
      api.why = "the run-time compiler (libnvrtc.so.13) could not be loaded";
      return;
    }
    bool all = true;
    auto get = [&](auto& fn, const char* sym) {
      fn = reinterpret_cast<std::remove_reference_t<decltype(fn)>>(dlsym(lib, sym));
      all = all && fn != nullptr;
    };
    get(api.version, "nvrtcVersion");
    get(api.create, "nvrtcCreateProgram");
    get(api.add_name, "nvrtcAddNameExpression");
    get(api.compile, "nvrtcCompileProgram");
    get(api.lowered, "nvrtcGetLoweredName");
    get(api.cubin_size, "nvrtcGetCUBINSize");
    get(api.cubin, "nvrtcGetCUBIN");
    get(api.log_size, "nvrtcGetProgramLogSize");
    get(api.log, "nvrtcGetProgramLog");
    get(api.destroy, "nvrtcDestroyProgram");
    get(api.error_string, "nvrtcGetErrorString");
    api.ok = all;
    if (!all) api.why = "libnvrtc lacks an expected entry point";
  });
  return api;
}

constexpr const char* kKernelExpr[2] = {
    "chemgb::k_integrate_plain<chemgb::Grp1, chemgb::SpecView, chemgb::SpecLayout>",
    "chemgb::k_integrate_persistent<chemgb::Grp1, chemgb::SpecView, chemgb::SpecLayout>"};
constexpr const char* kKernelTag[2] = {"plain", "persistent"};
// The library's own integration kernels are built with the same register cap.
constexpr const char* kOptions[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-maxrregcount=128"};
constexpr int kNumOptions = sizeof(kOptions) / sizeof(kOptions[0]);

uint64_t fnv1a(uint64_t h, const std::string& s) {
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

std::string cache_dir() {
  if (const char* e = std::getenv("CHEM_RTC_CACHE")) return e;
  Dl_info info{};
  if (dladdr(reinterpret_cast<void*>(&release_specialized), &info) && info.dli_fname) {
    std::string p = info.dli_fname;
    const size_t slash = p.rfind('/');
    if (slash != std::string::npos) return p.substr(0, slash) + "/rtc_cache";
  }
  return "";
}

bool read_file(const std::string& path, std::string& out) {
  std::ifstream f(path, std::ios::binary);
  if (!f) return false;
  std::ostringstream ss;
  ss << f.rdbuf();
  out = ss.str();
  return (bool)f || f.eof();
}

void write_file(const std::string& path, const std::string& data) {
  const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
  {
    std::ofstream f(tmp, std::ios::binary);
    if (!f) return;
    f.write(data.data(), (std::streamsize)data.size());
    if (!f) { std::remove(tmp.c_str()); return; }
  }
  std::rename(tmp.c_str(), path.c_str());   // atomic: readers see the old file or the whole new one
}

struct Compiled {
  std::string cubin, name, log;
  bool ok = false;
  bool cached = false;
};

void compile_one(const std::string& src, int which, const std::string& stem, Compiled& out) {
  if (!stem.empty() && read_file(stem + "_" + kKernelTag[which] + ".cubin", out.cubin) &&
      read_file(stem + "_" + kKernelTag[which] + ".name", out.name) && !out.cubin.empty() && !out.name.empty()) {
    out.ok = out.cached = true;
    return;
  }
  const Nvrtc& R = nvrtc();
  nvrtcProgram prog = nullptr;
  nvrtcResult r = R.create(&prog, src.c_str(), "chem_specialized.cu", kRtcHeaderCount, kRtcHeaderTexts,
                           kRtcHeaderNames);
  if (r != NVRTC_SUCCESS) { out.log = R.error_string(r); return; }
  r = R.add_name(prog, kKernelExpr[which]);
  if (r == NVRTC_SUCCESS) r = R.compile(prog, kNumOptions, kOptions);
  size_t ls = 0;
  if (R.log_size(prog, &ls) == NVRTC_SUCCESS && ls > 1) {
    out.log.resize(ls);
    R.log(prog, &out.log[0]);
    out.log.resize(ls - 1);
  }
  if (r == NVRTC_SUCCESS) {
    const char* lowered = nullptr;
    size_t cs = 0;
    r = R.lowered(prog, kKernelExpr[which], &lowered);
    if (r == NVRTC_SUCCESS) {
      out.name = lowered;
      r = R.cubin_size(prog, &cs);
    }
    if (r == NVRTC_SUCCESS) {
      out.cubin.resize(cs);
      r = R.cubin(prog, &out.cubin[0]);
    }
  }
  if (r != NVRTC_SUCCESS) {
    out.log = std::string(R.error_string(r)) + "\n" + out.log;
  } else {
    out.ok = true;
    if (!stem.empty()) {
      write_file(stem + "_" + kKernelTag[which] + ".cubin", out.cubin);
      write_file(stem + "_" + kKernelTag[which] + ".name", out.name);
    }
  }
  R.destroy(&prog);
}

}  // namespace

std::string specialized_source(const HostMech& hm, const CellLayout& L) {
  const HostProg& P = hm.prog[0];
  std::ostringstream s;
  s << "// mechanism-specialised integration kernels: n = " << hm.n << " species, R = " << hm.R << " reactions\n"
    << "#include \"integrate.cuh\"\n"
    << "namespace chemgb {\n"
    << "struct SpecView : MechView {\n"
    << "  static constexpr int width = " << P.width << ", n = " << hm.n << ", R = " << hm.R << ", m = " << hm.m
    << ", n_troe = " << hm.n_troe << ", n_tb = " << hm.n_tb << ", nY = " << hm.nY << ", nnz_S = " << hm.nnz_S
    << ", nnz_LU = " << hm.nnz_LU << ", n_dslot = " << hm.n_dslot << ";\n"
    << "  static constexpr int lu_steps = " << P.lu_kind.size() << ", sv_steps = " << P.sv_kind.size()
    << ", svT_steps = " << P.svT_kind.size() << ", n_jpass = " << hm.jpass.size() / 4 << ";\n"
    << "};\n"
    << "struct SpecLayout : CellLayout {\n"
    << "  static constexpr int y = " << L.y << ", ytmp = " << L.ytmp << ", f0 = " << L.f0 << ", U1 = " << L.U1
    << ", U2 = " << L.U2 << ", U3 = " << L.U3 << ", U4 = " << L.U4 << ", x = " << L.x << ", z = " << L.z
    << ", u = " << L.u << ", v = " << L.v << ";\n"
    << "  static constexpr int C = " << L.C << ", hRT = " << L.hRT << ", eg = " << L.eg << ", emg = " << L.emg
    << ", cpR = " << L.cpR << ", q = " << L.q << ", S = " << L.S << ", LU = " << L.LU << ", dinv = " << L.dinv
    << ", D = " << L.D << ", part = " << L.part << ", misc = " << L.misc << ", total = " << L.total << ";\n"
    << "};\n"
    << "static_assert(sizeof(SpecView) == sizeof(MechView) && sizeof(SpecLayout) == sizeof(CellLayout),\n"
    << "              \"the specialised views must keep the data members of the generic ones\");\n"
    << "}  // namespace chemgb\n";
  return s.str();
}

chem_status compile_specialized(const HostMech& hm, const CellLayout& L, bool load, SpecKernels& out,
                                std::string& err) {
  const Nvrtc& R = nvrtc();
  if (!R.ok) { err = R.why; return CHEM_EUNSUPPORTED; }
  const std::string src = specialized_source(hm, L);
  int major = 0, minor = 0;
  R.version(&major, &minor);
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(h, src);
  for (int i = 0; i < kRtcHeaderCount; ++i) h = fnv1a(fnv1a(h, kRtcHeaderNames[i]), kRtcHeaderTexts[i]);
  for (const char* o : kOptions) h = fnv1a(h, o);
  h = fnv1a(h, std::to_string(major) + "." + std::to_string(minor));
  std::string stem;
  const std::string dir = cache_dir();
  if (!dir.empty()) {
    mkdir(dir.c_str(), 0755);   // may exist already; an unwritable cache only costs the compile
    char hex[17];
    std::snprintf(hex, sizeof hex, "%016llx", (unsigned long long)h);
    stem = dir + "/" + hex;
  }
  const auto t0 = std::chrono::steady_clock::now();
  Compiled c[2];
  std::thread other(compile_one, std::cref(src), 1, std::cref(stem), std::ref(c[1]));
  compile_one(src, 0, stem, c[0]);
  other.join();
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < 2; ++i)
    if (!c[i].ok) {
      err = std::string("run-time compilation of the ") + kKernelTag[i] + " kernel failed: " + c[i].log;
      return CHEM_ECUDA;
    }
  SpecKernels k;
  k.from_cache = c[0].cached && c[1].cached;
  k.compile_s = k.from_cache ? 0.0 : secs;
  if (!load) {
    out.compile_s = k.compile_s;
    out.from_cache = k.from_cache;
    return CHEM_OK;
  }
  for (int i = 0; i < 2; ++i) {
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, c[i].cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    cudaKernel_t kern = nullptr;
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&kern, lib, c[i].name.c_str());
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (lib) cudaLibraryUnload(lib);
      release_specialized(k);
      err = std::string("loading the specialised ") + kKernelTag[i] + " kernel failed: " + cudaGetErrorString(e);
      return CHEM_ECUDA;
    }
    k.library[i] = lib;
    (i == 0 ? k.plain : k.persistent) = reinterpret_cast<const void*>(kern);
  }
  release_specialized(out);
  out = k;
  return CHEM_OK;
}

void release_specialized(SpecKernels& k) {
  for (void*& lib : k.library)
    if (lib) {
      cudaLibraryUnload(reinterpret_cast<cudaLibrary_t>(lib));
      lib = nullptr;
    }
  k.plain = k.persistent = nullptr;
}

}  // namespace chemgb
