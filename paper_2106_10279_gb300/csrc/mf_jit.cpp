// Run-time compilation of the generated process kernels for sm_103a (NVRTC)
// and loading them through the driver API, whose entry points are resolved at
// run time (no link-time dependency on the driver library, so the shared
// object loads on hosts without a GPU).  Compiled images are cached in the
// directory named by MF_JIT_CACHE (if set), keyed by a hash of the source,
// the options and the NVRTC version.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <cmath>
#include <map>
#include <mutex>
#include <sstream>

#include "mf_internal.h"

namespace {
#include "_embedded_sources.inc"   // kHeaderNames[], kHeaderSources[], kNumHeaders (from build.py)

uint64_t fnv1a(const std::string &s, uint64_t h = 1469598103934665603ull) {
    for (unsigned char c : s) { h ^= c; h *= 1099511628211ull; }
    return h;
}

std::mutex g_jit_mutex;

// NVRTC is opened by path with local symbol binding, so that the toolkit's
// compiler is used even when the process already holds another libnvrtc
// with the same soname (e.g. one bundled with a Python framework).
#ifndef MF_NVRTC_DEFAULT
#define MF_NVRTC_DEFAULT "libnvrtc.so.13"
#endif
struct Nvrtc {
    bool ok = false;
    std::string path;
    nvrtcResult (*version)(int *, int *);
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *, const char *const *);
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *);
    nvrtcResult (*log_size)(nvrtcProgram, size_t *);
    nvrtcResult (*log)(nvrtcProgram, char *);
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *);
    nvrtcResult (*cubin)(nvrtcProgram, char *);
    nvrtcResult (*destroy)(nvrtcProgram *);
};
Nvrtc g_nvrtc;

template <typename F>
bool sym(void *h, const char *name, F &fp) {
    fp = reinterpret_cast<F>(dlsym(h, name));
    return fp != nullptr;
}

bool open_nvrtc(std::string &err) {
    if (g_nvrtc.ok) return true;
    const char *env = std::getenv("MF_NVRTC_LIBRARY");
    const char *cands[] = {env && *env ? env : nullptr, MF_NVRTC_DEFAULT, "libnvrtc.so.13", "libnvrtc.so"};
    for (const char *c : cands) {
        if (!c) continue;
        void *h = dlopen(c, RTLD_NOW | RTLD_LOCAL);
        if (!h) { err += std::string(dlerror()) + "; "; continue; }
        Nvrtc n;
        if (sym(h, "nvrtcVersion", n.version) && sym(h, "nvrtcCreateProgram", n.create) &&
            sym(h, "nvrtcCompileProgram", n.compile) && sym(h, "nvrtcGetProgramLogSize", n.log_size) &&
            sym(h, "nvrtcGetProgramLog", n.log) && sym(h, "nvrtcGetCUBINSize", n.cubin_size) &&
            sym(h, "nvrtcGetCUBIN", n.cubin) && sym(h, "nvrtcDestroyProgram", n.destroy)) {
            n.ok = true;
            n.path = c;
            g_nvrtc = n;
            return true;
        }
        err += std::string(c) + ": missing symbols; ";
    }
    return false;
}
}  // namespace

namespace mfi {

mf_status jit_compile(const std::string &source, const std::string &name, std::vector<char> &cubin,
                      int ptxas_level) {
    std::lock_guard<std::mutex> lock(g_jit_mutex);
    std::string oerr;
    if (!open_nvrtc(oerr)) return fail(MF_EJIT, "cannot load NVRTC: " + oerr);
    std::vector<const char *> opts = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo",
                                      "--device-as-default-execution-space"};
    static const char *kLevels[4] = {"--ptxas-options=-O0", "--ptxas-options=-O1", "--ptxas-options=-O2",
                                     "--ptxas-options=-O3"};
    if (ptxas_level >= 0 && ptxas_level <= 2) opts.push_back(kLevels[ptxas_level]);
    const char *verbose = std::getenv("MF_JIT_VERBOSE");
    if (verbose && *verbose == '1') opts.push_back("--ptxas-options=-v");
    int vmaj = 0, vmin = 0;
    g_nvrtc.version(&vmaj, &vmin);
    std::string key = source;
    for (auto o : opts) key += o;
    for (int i = 0; i < kNumHeaders; ++i) key += kHeaderSources[i];
    key += std::to_string(vmaj) + "." + std::to_string(vmin);
    char hex[32];
    std::snprintf(hex, sizeof hex, "%016llx", (unsigned long long)fnv1a(key));
    // binaries compiled earlier in this process (keyed by the whole key text)
    static std::map<std::string, std::vector<char>> memo;
    auto hit = memo.find(key);
    if (hit != memo.end()) {
        cubin = hit->second;
        return MF_OK;
    }
    const char *dir = std::getenv("MF_JIT_CACHE");
    std::string path = dir && *dir ? std::string(dir) + "/mf_" + hex + ".cubin" : std::string();
    if (!path.empty()) {
        std::ifstream in(path, std::ios::binary);
        if (in) {
            cubin.assign(std::istreambuf_iterator<char>(in), std::istreambuf_iterator<char>());
            if (!cubin.empty()) {
                memo[key] = cubin;
                return MF_OK;
            }
        }
    }
    nvrtcProgram prog;
    if (g_nvrtc.create(&prog, source.c_str(), name.c_str(), kNumHeaders, kHeaderSources, kHeaderNames) !=
        NVRTC_SUCCESS)
        return fail(MF_EJIT, "nvrtcCreateProgram failed");
    nvrtcResult r = g_nvrtc.compile(prog, (int)opts.size(), opts.data());
    size_t log_size = 0;
    g_nvrtc.log_size(prog, &log_size);
    std::string log(log_size, '\0');
    if (log_size) g_nvrtc.log(prog, &log[0]);
    if (r != NVRTC_SUCCESS) {
        g_nvrtc.destroy(&prog);
        return fail(MF_EJIT, "NVRTC compilation of " + name + " failed: " + log);
    }
    if (verbose && *verbose == '1') std::fprintf(stderr, "[mf jit] %s (NVRTC %d.%d from %s)\n%s\n", name.c_str(), vmaj, vmin,
                     g_nvrtc.path.c_str(), log.c_str());
    size_t n = 0;
    g_nvrtc.cubin_size(prog, &n);
    cubin.resize(n);
    g_nvrtc.cubin(prog, cubin.data());
    g_nvrtc.destroy(&prog);
    memo[key] = cubin;
    if (!path.empty()) {
        std::string tmp = path + ".tmp" + std::to_string((long long)std::rand());
        std::ofstream out(tmp, std::ios::binary);
        out.write(cubin.data(), (std::streamsize)cubin.size());
        out.close();
        std::rename(tmp.c_str(), path.c_str());
    }
    return MF_OK;
}

// Driver-API entry points resolved at run time through the runtime (so the
// library has no link-time dependency on the driver library).
namespace {
struct DriverApi {
    bool ok = false;
    CUresult (*moduleLoadData)(CUmodule *, const void *) = nullptr;
    CUresult (*moduleUnload)(CUmodule) = nullptr;
    CUresult (*moduleGetFunction)(CUfunction *, CUmodule, const char *) = nullptr;
    CUresult (*funcGetAttribute)(int *, CUfunction_attribute, CUfunction) = nullptr;
    CUresult (*funcSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
    CUresult (*occupancy)(int *, CUfunction, int, size_t) = nullptr;
    CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                       CUstream, void **, void **) = nullptr;
    CUresult (*errorString)(CUresult, const char **) = nullptr;
};
DriverApi g_drv;
std::mutex g_drv_mutex;

template <typename F>
bool resolve(const char *name, F &fp) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    fp = reinterpret_cast<F>(p);
    return true;
}

mf_status driver() {
    std::lock_guard<std::mutex> lock(g_drv_mutex);
    if (g_drv.ok) return MF_OK;
    bool ok = resolve("cuModuleLoadData", g_drv.moduleLoadData) && resolve("cuModuleUnload", g_drv.moduleUnload) &&
              resolve("cuModuleGetFunction", g_drv.moduleGetFunction) &&
              resolve("cuFuncGetAttribute", g_drv.funcGetAttribute) &&
              resolve("cuFuncSetAttribute", g_drv.funcSetAttribute) &&
              resolve("cuOccupancyMaxActiveBlocksPerMultiprocessor", g_drv.occupancy) &&
              resolve("cuLaunchKernel", g_drv.launch) && resolve("cuGetErrorString", g_drv.errorString);
    if (!ok) return fail(MF_ECUDA, "cannot resolve the CUDA driver entry points");
    g_drv.ok = true;
    return MF_OK;
}

std::string drv_err(CUresult r) {
    const char *s = nullptr;
    if (g_drv.errorString) g_drv.errorString(r, &s);
    return s ? s : ("CUresult " + std::to_string((int)r));
}
}  // namespace

mf_status load_kernel(const std::vector<char> &cubin, Compiled &out, const char *name) {
    mf_status st = driver();
    if (st != MF_OK) return st;
    CUresult r = g_drv.moduleLoadData(&out.module, cubin.data());
    if (r != CUDA_SUCCESS) return fail(MF_ECUDA, "cuModuleLoadData: " + drv_err(r));
    r = g_drv.moduleGetFunction(&out.fn, out.module, name);
    if (r != CUDA_SUCCESS) return fail(MF_ECUDA, "cuModuleGetFunction: " + drv_err(r));
    // the flow kernel of a process module (absent in other modules)
    if (g_drv.moduleGetFunction(&out.fn_flow, out.module, "mf_flow_kernel") != CUDA_SUCCESS) out.fn_flow = nullptr;
    if (g_drv.moduleGetFunction(&out.fn_csamp, out.module, "mf_csamp_kernel") != CUDA_SUCCESS) out.fn_csamp = nullptr;
    for (CUfunction f : {out.fn_flow, out.fn_csamp})
        if (f && out.smem > 48 * 1024) g_drv.funcSetAttribute(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)out.smem);
    int regs = 0, local = 0;
    g_drv.funcGetAttribute(&regs, CU_FUNC_ATTRIBUTE_NUM_REGS, out.fn);
    g_drv.funcGetAttribute(&local, CU_FUNC_ATTRIBUTE_LOCAL_SIZE_BYTES, out.fn);
    out.regs = regs;
    out.local_bytes = (size_t)local;
    if (out.smem > 48 * 1024) {
        r = g_drv.funcSetAttribute(out.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)out.smem);
        if (r != CUDA_SUCCESS) return fail(MF_ECUDA, "cannot reserve dynamic shared memory: " + drv_err(r));
    }
    // shared-memory carve-out: just enough for every block the registers
    // allow on an SM, so that the rest stays L1 cache (the programs spill to
    // local memory, which lives there)
    int nb = 0, nb_regs = 0, stat = 0;
    g_drv.funcGetAttribute(&stat, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, out.fn);
    if (g_drv.occupancy(&nb_regs, out.fn, out.block, 0) == CUDA_SUCCESS && nb_regs > 0) {
        const double per_sm = (double)nb_regs * (double)(out.smem + (size_t)stat + 1024);
        // (a margin above the need: the driver picks a nearby supported size;
        // kernels that need most of the SM's shared memory ask for all of it)
        int pct = (int)std::ceil(100.0 * per_sm / (228.0 * 1024.0)) + 10;
        if (pct > 60) pct = 100;
        if (pct < 1) pct = 1;
        if (pct > 100) pct = 100;
        g_drv.funcSetAttribute(out.fn, CU_FUNC_ATTRIBUTE_PREFERRED_SHARED_MEMORY_CARVEOUT, pct);
    }
    r = g_drv.occupancy(&nb, out.fn, out.block, out.smem);
    if (r != CUDA_SUCCESS || nb < 1) return fail(MF_ECUDA, "process kernel cannot be resident on an SM");
    out.max_blocks_per_sm = nb;
    return MF_OK;
}

void unload_kernel(Compiled &k) {
    if (k.module && g_drv.ok) g_drv.moduleUnload(k.module);
    k.module = nullptr;
    k.fn = nullptr;
    k.fn_flow = nullptr;
    k.fn_csamp = nullptr;
}

mf_status launch_kernel(const Compiled &k, unsigned grid, void **args, cudaStream_t s, int variant) {
    CUfunction f = variant == 1 ? k.fn_flow : variant == 2 ? k.fn_csamp : k.fn;
    if (!f) return fail(MF_EUNSUPPORTED, "the process module has no kernel of this variant");
    CUresult r = g_drv.launch(f, grid, 1, 1, (unsigned)k.block, 1, 1, (unsigned)k.smem, (CUstream)s, args, nullptr);
    if (r != CUDA_SUCCESS) return fail(MF_ECUDA, "process kernel launch: " + drv_err(r));
    return MF_OK;
}

}  // namespace mfi
