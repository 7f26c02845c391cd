// user_kernel.cu -- sweeps for a user kernel G(r), compiled at run time.
//
// The treecode needs only evaluations of G (Sec. I; Sec. V names other kernels as the
// method's reach), so besides the built-in Coulomb and Yukawa kernels (Eq. 2) a context can
// register any smooth, non-oscillatory radial kernel as CUDA source.  The library compiles
// the device code of its own sweeps (sweep_device.cuh, embedded in the library at build
// time) together with the user's two functions, with NVRTC, and keeps the resulting module
// in the context.  NVRTC is loaded with dlopen on first use, so the library itself does not
// depend on it.
#include <dlfcn.h>

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"
#include "sweep_device.cuh"

namespace bltc {

extern const char* const kSweepDeviceSource;   // sweep_device.cuh, generated by build.py

namespace {

// The NVRTC entry points used here (nvrtc.h declares them with an opaque program handle and
// an int-sized result enum).
struct Nvrtc {
    void* h = nullptr;
    int (*create)(void**, const char*, const char*, int, const char* const*, const char* const*) = nullptr;
    int (*compile)(void*, int, const char* const*) = nullptr;
    int (*log_size)(void*, size_t*) = nullptr;
    int (*log)(void*, char*) = nullptr;
    int (*cubin_size)(void*, size_t*) = nullptr;
    int (*cubin)(void*, char*) = nullptr;
    int (*destroy)(void**) = nullptr;
};

const Nvrtc* nvrtc() {
    static std::once_flag once;
    static Nvrtc n;
    std::call_once(once, [] {
        std::vector<std::string> cands;
        if (const char* p = std::getenv("BLTC_NVRTC_PATH")) cands.push_back(p);
        if (const char* p = std::getenv("CUDA_HOME")) cands.push_back(std::string(p) + "/lib64/libnvrtc.so");
        cands.push_back("libnvrtc.so.13");
        cands.push_back("libnvrtc.so");
        cands.push_back("/usr/local/cuda/lib64/libnvrtc.so");
        for (const std::string& c : cands) {
            void* h = dlopen(c.c_str(), RTLD_NOW | RTLD_LOCAL);
            if (!h) continue;
            Nvrtc t;
            t.h = h;
            t.create = reinterpret_cast<decltype(t.create)>(dlsym(h, "nvrtcCreateProgram"));
            t.compile = reinterpret_cast<decltype(t.compile)>(dlsym(h, "nvrtcCompileProgram"));
            t.log_size = reinterpret_cast<decltype(t.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
            t.log = reinterpret_cast<decltype(t.log)>(dlsym(h, "nvrtcGetProgramLog"));
            t.cubin_size = reinterpret_cast<decltype(t.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
            t.cubin = reinterpret_cast<decltype(t.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
            t.destroy = reinterpret_cast<decltype(t.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
            if (t.create && t.compile && t.log_size && t.log && t.cubin_size && t.cubin && t.destroy) {
                n = t;
                return;
            }
            dlclose(h);
        }
    });
    return n.h ? &n : nullptr;
}

// What the embedded device code expects from the host headers, restated for NVRTC (which
// sees no system headers), then the user's functions, the sweep code, and two entry points
// with C names.
std::string module_source(const char* user) {
    std::string s;
    s += "typedef signed char int8_t;\ntypedef unsigned char uint8_t;\n";
    s += "typedef int int32_t;\ntypedef unsigned int uint32_t;\n";
    s += "typedef long long int64_t;\ntypedef unsigned long long uint64_t;\n";
    s += "enum { BLTC_KERNEL_COULOMB = " + std::to_string(BLTC_KERNEL_COULOMB) +
         ", BLTC_KERNEL_YUKAWA = " + std::to_string(BLTC_KERNEL_YUKAWA) + " };\n";
    s += "#define BLTC_MAX_DEGREE " + std::to_string(BLTC_MAX_DEGREE) + "\n";
    s += "#define BLTC_NVRTC 1\n";
    s += "namespace bltc { struct __align__(32) D4 { double x, y, z, w; }; }\n";
    s += "#line 1 \"user_kernel\"\n";
    s += user;
    s += "\n#line 1 \"sweep_device.cuh\"\n";
    s += kSweepDeviceSource;
    s += "\nextern \"C\" __global__ void __launch_bounds__(bltc::sweepdev::kThreads, bltc::sweepdev::kMinBlocks)\n"
         "bltc_user_sweep_mixed(bltc::sweepdev::SweepArgs a) {\n"
         "    bltc::sweepdev::sweep_mixed_body<bltc::sweepdev::kKerUser>(a);\n}\n"
         "extern \"C\" __global__ void __launch_bounds__(bltc::sweepdev::kThreads, 2)\n"
         "bltc_user_sweep_fp64(bltc::sweepdev::SweepArgs a) {\n"
         "    bltc::sweepdev::sweep_fp64_body<bltc::sweepdev::kKerUser>(a);\n}\n";
    return s;
}

}  // namespace

bool compile_user_kernel(const char* source, int arch, std::string* log, std::vector<char>* cubin) {
    const Nvrtc* nv = nvrtc();
    if (!nv) throw Error(BLTC_ERR_STATE, "user kernel: NVRTC (libnvrtc.so) not found; set BLTC_NVRTC_PATH");
    require(source != nullptr, "user kernel: NULL source");
    require(arch >= 50 && arch < 1000, "user kernel: bad architecture");
    const std::string src = module_source(source);
    void* prog = nullptr;
    if (nv->create(&prog, src.c_str(), "bltc_user_module.cu", 0, nullptr, nullptr) != 0)
        throw Error(BLTC_ERR_CUDA, "user kernel: nvrtcCreateProgram failed");
    // architecture-specific targets (sm_90a and later) expose every feature the sweeps use
    const std::string a = "--gpu-architecture=sm_" + std::to_string(arch) + (arch >= 90 ? "a" : "");
    const char* opts[] = {a.c_str(), "-std=c++17", "-default-device"};
    const bool ok = nv->compile(prog, 3, opts) == 0;
    size_t n = 0;
    nv->log_size(prog, &n);
    if (log) {
        log->assign(n, '\0');
        if (n) nv->log(prog, &(*log)[0]);
        while (!log->empty() && log->back() == '\0') log->pop_back();
    }
    if (ok && cubin) {
        size_t m = 0;
        nv->cubin_size(prog, &m);
        cubin->resize(m);
        if (m) nv->cubin(prog, cubin->data());
    }
    nv->destroy(&prog);
    return ok;
}

int register_user_kernel(Context* c, const char* source) {
    int major = 0, minor = 0;
    BLTC_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device));
    BLTC_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, c->device));
    std::string log;
    std::vector<char> cubin;
    if (!compile_user_kernel(source, major * 10 + minor, &log, &cubin))
        throw Error(BLTC_ERR_ARG, "user kernel: compilation failed:\n" + log);
    Context::UserKernel k;
    BLTC_CUDA(cudaLibraryLoadData(&k.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
    try {
        BLTC_CUDA(cudaLibraryGetKernel(&k.mixed, k.lib, "bltc_user_sweep_mixed"));
        BLTC_CUDA(cudaLibraryGetKernel(&k.fp64, k.lib, "bltc_user_sweep_fp64"));
        BLTC_CUDA(cudaKernelSetAttributeForDevice(k.mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  sweepdev::kMixedSmem, c->device));
    } catch (...) {
        cudaLibraryUnload(k.lib);
        throw;
    }
    c->user_kernels.push_back(k);
    return BLTC_KERNEL_USER_BASE + static_cast<int>(c->user_kernels.size()) - 1;
}

}  // namespace bltc
