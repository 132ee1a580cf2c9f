// lbm_jit.h -- run-time compilation of generated CUDA C++ for sm_103a.
//
// The adjoint engine turns the recorded tape of a step into straight-line
// level kernels (one per level and direction) and compiles them once per
// tape structure with NVRTC straight to an sm_103a cubin, loaded with
// cudaLibraryLoadData.  NVRTC is opened at run time, so the library keeps
// no link dependency on it; when it cannot be opened or a compilation fails
// the caller falls back to its interpreter and reason() says why.
// LBM_JIT_DUMP=<path> in the environment writes each generated source there.
#pragma once

#include <cuda_runtime.h>
#include <dlfcn.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

namespace lbm_jit {

// The NVRTC entry points used here, with the types of nvrtc.h.
typedef int nvrtcResult_t;
typedef struct _nvrtcProgram *nvrtcProgram_t;
struct Nvrtc {
    nvrtcResult_t (*create)(nvrtcProgram_t *, const char *, const char *, int, const char *const *,
                            const char *const *) = nullptr;
    nvrtcResult_t (*compile)(nvrtcProgram_t, int, const char *const *) = nullptr;
    nvrtcResult_t (*log_size)(nvrtcProgram_t, size_t *) = nullptr;
    nvrtcResult_t (*log)(nvrtcProgram_t, char *) = nullptr;
    nvrtcResult_t (*cubin_size)(nvrtcProgram_t, size_t *) = nullptr;
    nvrtcResult_t (*cubin)(nvrtcProgram_t, char *) = nullptr;
    nvrtcResult_t (*destroy)(nvrtcProgram_t *) = nullptr;
    bool ok = false;
    std::string why;
};

inline std::string &reason()
{
    static std::string r;
    return r;
}

inline Nvrtc &nvrtc()
{
    static Nvrtc N;
    static bool tried = false;
    if (tried) return N;
    tried = true;
    const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void *h = nullptr;
    for (const char *n : names)
        if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) {
        N.why = "libnvrtc could not be opened";
        return N;
    }
    auto sym = [&](auto &f, const char *name) {
        f = reinterpret_cast<std::remove_reference_t<decltype(f)>>(dlsym(h, name));
        return f != nullptr;
    };
    N.ok = sym(N.create, "nvrtcCreateProgram") && sym(N.compile, "nvrtcCompileProgram") &&
           sym(N.log_size, "nvrtcGetProgramLogSize") && sym(N.log, "nvrtcGetProgramLog") &&
           sym(N.cubin_size, "nvrtcGetCUBINSize") && sym(N.cubin, "nvrtcGetCUBIN") &&
           sym(N.destroy, "nvrtcDestroyProgram");
    if (!N.ok) N.why = "libnvrtc lacks an entry point";
    return N;
}

// The loaded library of a source on the current device, compiled on first
// request; nullptr (and reason() set) on failure.  Serialised by one lock, so
// handles used from several threads share the cache safely.
inline cudaLibrary_t library(const std::string &src)
{
    static std::map<std::pair<int, std::string>, cudaLibrary_t> cache;
    static std::mutex lock;
    std::lock_guard<std::mutex> guard(lock);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    auto key = std::make_pair(dev, src);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    if (const char *dump = getenv("LBM_JIT_DUMP")) {   // the generated source, for reading
        if (FILE *f = fopen(dump, "w")) {
            fputs(src.c_str(), f);
            fclose(f);
        }
    }
    Nvrtc &N = nvrtc();
    if (!N.ok) {
        reason() = N.why;
        return nullptr;
    }
    nvrtcProgram_t prog = nullptr;
    if (N.create(&prog, src.c_str(), "lbm_adjoint_levels.cu", 0, nullptr, nullptr) != 0) {
        reason() = "nvrtcCreateProgram failed";
        return nullptr;
    }
    const char *opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device"};
    const int rc = N.compile(prog, 3, opts);
    std::vector<char> cubin;
    if (rc == 0) {
        size_t n = 0;
        N.cubin_size(prog, &n);
        cubin.resize(n);
        N.cubin(prog, cubin.data());
    } else {
        size_t n = 0;
        N.log_size(prog, &n);
        std::string log(n, '\0');
        N.log(prog, &log[0]);
        reason() = "NVRTC compilation failed: " + log.substr(0, 400);
    }
    N.destroy(&prog);
    if (cubin.empty()) return nullptr;
    cudaLibrary_t lib = nullptr;
    if (cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess) {
        cudaGetLastError();
        reason() = "cudaLibraryLoadData failed";
        return nullptr;
    }
    cache[key] = lib;
    return lib;
}

}  // namespace lbm_jit
