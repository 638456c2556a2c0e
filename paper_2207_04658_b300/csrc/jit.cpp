// jit.cpp -- the step kernel specialised to one scheme.  step_kernels.cuh is compiled at run
// time by NVRTC with the scene's codec table (Sec. 3.1 Eq. 3, Sec. 7 bit pack) as
// compile-time constants (QMPM_SPECIALIZED_CODEC), with the record's word count and the
// dither flag (FP32 state: the word count alone), loaded as a CUDA library and launched by
// launch_g2p2g in place of the kernel compiled with the library.  The arithmetic is the
// same; what changes is that a component's word index, shift and straddle are immediates,
// so the decode reads fixed shared-memory offsets and the encode assembles the record words
// in registers.  Compiled cubins are kept for the life of the process, one per generated
// source (that is, per dimension, material, statistics and dither flags and codec table).
#include <dlfcn.h>
#include <nvrtc.h>

#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "qmpm_internal.h"

namespace qmpm {
namespace {

struct Compiled {
    std::vector<char> cubin;
    std::string lowered;   // the kernel instance's symbol in the cubin
    double seconds = 0.0;  // NVRTC compile time of the first build
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
};

std::mutex g_mu;
std::map<std::string, Compiled> g_cache;

// Directory of this library: the kernel sources sit in csrc/ beside it.
std::string lib_dir()
{
    Dl_info info;
    if (!dladdr(reinterpret_cast<void *>(&lib_dir), &info) || !info.dli_fname) return ".";
    const std::string p(info.dli_fname);
    const size_t k = p.rfind('/');
    return k == std::string::npos ? std::string(".") : p.substr(0, k);
}

// A float as an exact C++17 hexadecimal literal.
std::string hex_float(float v)
{
    char b[64];
    std::snprintf(b, sizeof b, "%af", (double)v);
    return b;
}

std::string kernel_name(int dim, int material, bool quant, bool stats)
{
    return "qmpm::step_kernel<" + std::to_string(dim) + ", " + std::to_string(material) + ", " +
           (quant ? "true" : "false") + ", " + (stats ? "true" : "false") + ", true>";
}

// cc == nullptr: FP32 state (the word count and the dither flag only)
std::string kernel_source(int dim, int material, int W, bool dither, const CompCodec *cc, int nc)
{
    std::string s;
    s += "#define QMPM_SPECIALIZED_CODEC 1\n";
    s += "#include \"qmpm_internal.h\"\n";
    s += "namespace qmpm {\n";
    s += "constexpr int kSpecDim = " + std::to_string(dim) + ", kSpecMat = " + std::to_string(material) +
         ", kSpecWords = " + std::to_string(W) + ";\n";
    s += std::string("constexpr bool kSpecQuant = ") + (cc ? "true" : "false") + ", kSpecDither = " +
         (dither ? "true" : "false") + ";\n";
    if (!cc) {
        s += "__device__ constexpr CompCodec kSpecCodec[1] = {};\n}  // namespace qmpm\n";
        s += "#include \"step_kernels.cuh\"\n";
        return s;
    }
    s += "__device__ constexpr CompCodec kSpecCodec[" + std::to_string(nc) + "] = {\n";
    for (int c = 0; c < nc; ++c) {
        const CompCodec &k = cc[c];
        s += "    {" + std::to_string(k.word) + ", " + std::to_string(k.shift) + ", " + std::to_string(k.straddle) +
             ", " + std::to_string(k.mask) + "u, " + std::to_string(k.offset) + ", " + std::to_string(k.umax) +
             "u, " + hex_float(k.enc_scale) + ", " + hex_float(k.dec_scale) + ", " + hex_float(k.dec_bias) + ", " +
             std::to_string(k.field) + "},\n";
    }
    s += "};\n}  // namespace qmpm\n";
    s += "#include \"step_kernels.cuh\"\n";
    return s;
}

int nvrtc_fail(nvrtcResult r, const char *what, std::string &err)
{
    err = std::string("specialised step kernel: ") + what + ": " + nvrtcGetErrorString(r);
    return QMPM_ERR_CUDA;
}

// Compiles src (the cubin for sm_103a; no device needed) into out.
int compile(const std::string &src, const std::string &name, Compiled &out, std::string &err)
{
    nvrtcProgram prog = nullptr;
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "qmpm_specialized_step.cu", 0, nullptr, nullptr);
    if (r != NVRTC_SUCCESS) return nvrtc_fail(r, "create", err);
    r = nvrtcAddNameExpression(prog, name.c_str());
    if (r != NVRTC_SUCCESS) {
        nvrtcDestroyProgram(&prog);
        return nvrtc_fail(r, "name expression", err);
    }
    const std::string inc = "-I" + lib_dir() + "/csrc";
    // the library's own flags where NVRTC has them; unannotated (constexpr) helpers and the
    // C ABI's declarations are taken as device declarations
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", inc.c_str(), "-lineinfo", "-default-device"};
    const auto t0 = std::chrono::steady_clock::now();
    r = nvrtcCompileProgram(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
    out.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        std::string log;
        if (nvrtcGetProgramLogSize(prog, &n) == NVRTC_SUCCESS && n > 1) {
            log.resize(n);
            nvrtcGetProgramLog(prog, &log[0]);
            if (log.size() > 2000) log = "..." + log.substr(log.size() - 2000);
        }
        nvrtcDestroyProgram(&prog);
        err = std::string("specialised step kernel: compile: ") + nvrtcGetErrorString(r) + "\n" + log;
        return QMPM_ERR_CUDA;
    }
    const char *lowered = nullptr;
    r = nvrtcGetLoweredName(prog, name.c_str(), &lowered);
    if (r == NVRTC_SUCCESS && lowered) out.lowered = lowered;
    size_t n = 0;
    if (r == NVRTC_SUCCESS) r = nvrtcGetCUBINSize(prog, &n);
    if (r == NVRTC_SUCCESS) {
        out.cubin.resize(n);
        r = nvrtcGetCUBIN(prog, out.cubin.data());
    }
    nvrtcDestroyProgram(&prog);
    if (r != NVRTC_SUCCESS || out.lowered.empty()) return nvrtc_fail(r, "cubin", err);
    return QMPM_OK;
}

// The cache entry of this codec, compiled on first use.  g_mu held.
int entry(int dim, int material, bool stats, int W, bool dither, const CompCodec *cc, int nc, Compiled *&out,
          std::string &err)
{
    const std::string src = kernel_source(dim, material, W, dither, cc, nc);
    const std::string name = kernel_name(dim, material, cc != nullptr, stats);
    const std::string key = name + "\n" + src;
    auto it = g_cache.find(key);
    if (it == g_cache.end()) {
        Compiled c;
        const int rc = compile(src, name, c, err);
        if (rc != QMPM_OK) return rc;
        it = g_cache.emplace(key, std::move(c)).first;
    }
    out = &it->second;
    return QMPM_OK;
}

}  // namespace

int specialize_step_kernel(Ctx &c, std::string &err)
{
    const bool stats = (c.scene.flags & QMPM_FLAG_STATS) != 0;
    std::lock_guard<std::mutex> lk(g_mu);
    Compiled *e = nullptr;
    int rc = entry(c.scene.dim, c.scene.material, stats, c.W, c.scene.dither != 0, c.quant ? c.cc : nullptr,
                   c.n_comp, e, err);
    if (rc != QMPM_OK) return rc;
    if (!e->kern) {
        cudaError_t r = cudaLibraryLoadData(&e->lib, e->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
        if (r == cudaSuccess) r = cudaLibraryGetKernel(&e->kern, e->lib, e->lowered.c_str());
        if (r != cudaSuccess) {
            cudaGetLastError();
            if (e->lib) cudaLibraryUnload(e->lib);
            e->lib = nullptr;
            e->kern = nullptr;
            err = std::string("specialised step kernel: load: ") + cudaGetErrorString(r);
            return QMPM_ERR_CUDA;
        }
    }
    c.spec_kernel = reinterpret_cast<void *>(e->kern);
    c.spec_seconds = e->seconds;
    c.spec_smem = 0;
    c.spec_per_sm = 0;
    return QMPM_OK;
}

int specialize_compile_only(int dim, int material, bool stats, bool dither, int W, const CompCodec *cc, int nc,
                            double *seconds, int64_t *cubin_bytes, std::string &err)
{
    std::lock_guard<std::mutex> lk(g_mu);
    Compiled *e = nullptr;
    const int rc = entry(dim, material, stats, W, dither, cc, nc, e, err);
    if (rc != QMPM_OK) return rc;
    if (seconds) *seconds = e->seconds;
    if (cubin_bytes) *cubin_bytes = (int64_t)e->cubin.size();
    return QMPM_OK;
}

cudaError_t launch_specialized(Ctx &c, const StepParams &p)
{
    const void *k = c.spec_kernel;
    const size_t smem = step_smem_bytes(c.scene.dim, c.W);
    if (c.spec_smem != smem) {
        // persistent grid: as many CTAs as fit on every SM at once, as for the generic kernel
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
        if (e != cudaSuccess) return e;
        c.spec_per_sm = per_sm > 0 ? per_sm : 1;
        c.spec_smem = smem;
    }
    StepParams q = p;
    void *args[] = {&q};
    return cudaLaunchKernel(k, dim3((unsigned)(c.n_sms * c.spec_per_sm)), dim3(kThreads), args, smem, c.stream);
}

}  // namespace qmpm
