// Run-time specialisation of the lane-group FP32 integrator for one network.
//
// The lane-group kernel (integrate_grp.cuh) reads its row layout (node rows
// per lane, positions per row) from the launch arguments, so every row costs
// a loop with run-time bounds.  For a fixed network the layout is known when
// the handle is created; this file compiles a kernel with the layout as
// compile-time constants with NVRTC for sm_103a, loads the cubin with the
// CUDA runtime's library API and launches it.  Two kernels can be compiled:
//   * register records (integrate_rr.cuh, the default): every lane keeps its
//     edge records in registers, one shared load per edge;
//   * shared records (integrate_grp.cuh with the layout fixed): the same
//     source as the run-time-layout kernel, used when the register records
//     would not fit (a lane with many edge positions) or on request.
// Compiled kernels are cached per process by their source text, so handles
// of the same network share one compile.
//
// libnvrtc is opened with dlopen: a machine without it, or a failed compile,
// leaves the run-time-layout kernel in charge (GRINS_JIT=0 forces that).
#include <dlfcn.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvJitLink.h>
#include <nvrtc.h>

#include "integrate_grp.cuh"

namespace grins {

namespace {

// Kernel sources embedded at build time (jit_sources.inc, generated by
// build.py from the files of this folder and include/).
#include "jit_sources.inc"

// C integer types for the run-time compile (grins_racipe.h includes
// <stdint.h>, which NVRTC does not ship).
const char *const kStdintStandIn =
    "#pragma once\n"
    "typedef signed char int8_t; typedef unsigned char uint8_t;\n"
    "typedef short int16_t; typedef unsigned short uint16_t;\n"
    "typedef int int32_t; typedef unsigned int uint32_t;\n"
    "typedef long long int64_t; typedef unsigned long long uint64_t;\n"
    "typedef unsigned long long uintptr_t;\n";

struct NvrtcApi {
    bool ok = false;
    std::string why;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcGetErrorString) err = nullptr;
};

NvrtcApi &nvrtc()
{
    static NvrtcApi api;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *n : names)
            if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) { api.why = "libnvrtc not found"; return; }
        api.create = reinterpret_cast<decltype(api.create)>(dlsym(h, "nvrtcCreateProgram"));
        api.compile = reinterpret_cast<decltype(api.compile)>(dlsym(h, "nvrtcCompileProgram"));
        api.log_size = reinterpret_cast<decltype(api.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
        api.log = reinterpret_cast<decltype(api.log)>(dlsym(h, "nvrtcGetProgramLog"));
        api.cubin_size = reinterpret_cast<decltype(api.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
        api.cubin = reinterpret_cast<decltype(api.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
        api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
        api.err = reinterpret_cast<decltype(api.err)>(dlsym(h, "nvrtcGetErrorString"));
        api.ok = api.create && api.compile && api.log_size && api.log && api.cubin_size && api.cubin &&
                 api.destroy && api.err;
        if (!api.ok) api.why = "libnvrtc lacks an expected symbol";
    });
    return api;
}

constexpr int kJitWarps = 4;         // warps per block of the shared-record kernel

// Warps per block of a register-record kernel: 4, or GRINS_JIT_WARPS (1, 2,
// 4 or 8; a tuning knob -- the kernel's warps are independent, so the block
// size only sets the granularity of residency).
int jit_warps(int kind)
{
    if (kind == kJitShared) return kJitWarps;
    if (const char *ev = std::getenv("GRINS_JIT_WARPS")) {
        const int w = std::atoi(ev);
        if (w == 1 || w == 2 || w == 4 || w == 8) return w;
    }
    return kJitWarps;
}

// One cache entry: a kernel for one (layout, kind), compiled once per
// process, in the calling thread or in the background pool.
struct JitEntry {
    std::atomic<int> state{0};   // 0 compiling, 1 ready, -1 failed
    std::string why;
    int kind = kJitShared;
    int warps = kJitWarps;       // warps per block
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
};

// Result of one NVRTC compile and load (the compile log's spill count
// decides whether a register-record kernel is compiled again with fewer
// resident blocks).
struct JitBuild {
    bool ok = false;
    std::string why;
    int spill_bytes = 0;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
};

// Cache and background pool.  Both are created once and never destroyed:
// a pool thread may still be compiling when the process exits.
struct JitCache {
    std::mutex mu;
    std::condition_variable cv;            // an entry left the compiling state
    std::map<std::string, std::shared_ptr<JitEntry>> map;
};
JitCache &jit_cache()
{
    static JitCache *c = new JitCache();
    return *c;
}

struct JitPool {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::function<void()>> tasks;
    int threads = 0;
};
JitPool &jit_pool()
{
    static JitPool *p = new JitPool();
    return *p;
}

// Runs f on a pool thread; the pool grows to (cores - 2) threads, at least
// one, as tasks arrive.
void jit_pool_push(std::function<void()> f)
{
    JitPool &p = jit_pool();
    std::lock_guard<std::mutex> lock(p.mu);
    p.tasks.push_back(std::move(f));
    const int cores = (int)std::thread::hardware_concurrency();
    const int cap = cores > 3 ? cores - 2 : 1;
    if (p.threads < cap && (int)p.tasks.size() > 0) {
        ++p.threads;
        std::thread([&p] {
            std::unique_lock<std::mutex> l(p.mu);
            for (;;) {
                p.cv.wait(l, [&p] { return !p.tasks.empty(); });
                std::function<void()> t = std::move(p.tasks.front());
                p.tasks.pop_front();
                l.unlock();
                t();
                l.lock();
            }
        }).detach();
    }
    p.cv.notify_one();
}

// Register cap of a register-record kernel: 0 (residency from the block
// count, __launch_bounds__), or GRINS_JIT_MAXNREG (64..255, __maxnreg__; a
// tuning knob -- caps between the launch-bounds steps).
int jit_maxnreg(int kind)
{
    if (kind == kJitShared) return 0;
    if (const char *ev = std::getenv("GRINS_JIT_MAXNREG")) {
        const int r = std::atoi(ev);
        if (r >= 64 && r <= 255) return r;
    }
    return 0;
}

// The row layout of g as compile-time constants (kGrpCtRows, GrpRowCt<r>)
// in the current namespace of the generated source.
std::string layout_prelude(const GrpTopo &g, bool links)
{
    std::string s;
    char buf[256];
    std::snprintf(buf, sizeof(buf), "constexpr int kGrpCtRows = %d;\n", g.R);
    s += buf;
    s += "template <int r> struct GrpRowCt { static constexpr int off = 0, deg = 0, link = -1; };\n";
    for (int r = 0; r < g.R; ++r) {
        std::snprintf(buf, sizeof(buf),
                      "template <> struct GrpRowCt<%d> { static constexpr int off = %d, deg = %d, link = %d; };\n",
                      r, g.row_off[r], g.row_deg[r], links ? g.link_to[r] : -1);
        s += buf;
    }
    return s;
}

// Generated prelude + kernel wrapper for one layout.
std::string jit_main(const GrpTopo &g, int kind, int minb, int warps, int method)
{
    std::string s;
    char buf[256];
    s += "#define GRINS_GRP_CT 1\n";
#ifdef GRINS_CHECKED
    s += "#define GRINS_CHECKED 1\n";
#endif
    if (kind == kJitShared) {
#ifdef GRINS_GRP_ROLL_STAGES
        s += "#define GRINS_GRP_ROLL_STAGES 1\n";
#else
        // unrolled stages repeat the right-hand side seven times: keep the
        // stage loop when a lane's edge list is long (the code would outgrow
        // the instruction cache)
        if (g.P > 32) s += "#define GRINS_GRP_ROLL_STAGES 1\n";
#endif
    }
    s += "#include \"common.cuh\"\nnamespace grins {\n";
    s += layout_prelude(g, kind != kJitShared);
    if (kind != kJitShared) {
        s += "}\n#include \"integrate_rr.cuh\"\n";
        char bounds[64];
        if (const int mr = jit_maxnreg(kind)) std::snprintf(bounds, sizeof(bounds), "__maxnreg__(%d)", mr);
        else std::snprintf(bounds, sizeof(bounds), "__launch_bounds__(%d, %d)", warps * kWarp, minb);
        std::snprintf(buf, sizeof(buf),
                      "extern \"C\" __global__ void %s grins_grp_ct(const grins::IntegrateArgs a)\n"
                      "{\n    grins::rr_body<%d, %d, %d, %s, %d, %s, %s, %s>(a);\n}\n",
                      bounds, g.R, warps, g.L,
                      kind == kJitRegisters64 ? "double" : (kind == kJitRegistersDD ? "grins::dd" : "float"),
                      method & kJitMethodMask,
                      (method & kJitSeries) ? "true" : "false", (method & kJitTail) ? "true" : "false",
                      (method & kJitCancel) ? "true" : "false");
    } else {
        s += "}\n#include \"integrate_grp.cuh\"\n";
        std::snprintf(buf, sizeof(buf),
                      "extern \"C\" __global__ void __launch_bounds__(%d, %d) grins_grp_ct(const grins::IntegrateArgs a)\n"
                      "{\n    grins::grp_body<%d, %d, %d, %d>(a);\n}\n",
                      kJitWarps * kWarp, minb, g.R, kJitWarps, g.L, g.R);
    }
    s += buf;
    return s;
}

// Spill bytes reported by ptxas in a compile log ("N bytes spill stores").
int log_spill_bytes(const std::string &log)
{
    int total = 0;
    for (size_t p = log.find(" bytes spill stores"); p != std::string::npos;
         p = log.find(" bytes spill stores", p + 1)) {
        size_t b = p;
        while (b > 0 && log[b - 1] >= '0' && log[b - 1] <= '9') --b;
        if (b < p) total += std::atoi(log.substr(b, p - b).c_str());
    }
    return total;
}

JitBuild jit_compile(const std::string &src, const char *kname = "grins_grp_ct")
{
    JitBuild b;
    NvrtcApi &api = nvrtc();
    if (!api.ok) { b.why = api.why; return b; }
    std::vector<const char *> hdr_src, hdr_name;
    for (int i = 0; i < kJitSourceCount; ++i) {
        hdr_src.push_back(kJitSources[i]);
        hdr_name.push_back(kJitSourceNames[i]);
    }
    hdr_src.push_back(kStdintStandIn);
    hdr_name.push_back("stdint.h");
    nvrtcProgram prog = nullptr;
    nvrtcResult r = api.create(&prog, src.c_str(), "grins_grp_ct.cu", (int)hdr_src.size(), hdr_src.data(),
                               hdr_name.data());
    if (r != NVRTC_SUCCESS) { b.why = std::string("nvrtcCreateProgram: ") + api.err(r); return b; }
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo", "-default-device",
                          "--ptxas-options=-v"};
    r = api.compile(prog, 5, opts);
    size_t n = 0;
    api.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) api.log(prog, &log[0]);
    if (r != NVRTC_SUCCESS) {
        b.why = std::string("nvrtcCompileProgram: ") + api.err(r) + "\n" + log;
        api.destroy(&prog);
        return b;
    }
    b.spill_bytes = log_spill_bytes(log);
    n = 0;
    api.cubin_size(prog, &n);
    std::vector<char> cubin(n);
    api.cubin(prog, cubin.data());
    api.destroy(&prog);
    cudaError_t ce = cudaLibraryLoadData(&b.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&b.kern, b.lib, kname);
    if (ce != cudaSuccess) { b.why = std::string("loading the compiled kernel: ") + cudaGetErrorString(ce); return b; }
    b.ok = true;
    return b;
}

// Minimum resident blocks per SM for a kernel of this kind and layout: for
// register records from the estimate of a lane's registers (about 4 per edge
// position and 11 per row on top of ~40; ptxas usually fits a little more
// than the estimate, and a spilling compile is retried with one block
// fewer).  Counted in blocks of 4 warps and scaled to the kernel's block
// size; GRINS_JIT_MINB overrides it in blocks of that size (a tuning knob).
int jit_minb(const GrpTopo &g, int kind)
{
    const int est = 4 * g.P + 11 * g.R + 40;
    int minb = kind == kJitRegisters ? (est <= 144 ? 4 : (est <= 176 ? 3 : 2)) : GRINS_GRP_MINB;
    if (kind == kJitRegisters64) {          // 2 registers per value, 5 per position
        const int est64 = 5 * g.P + 22 * g.R + 60;
        minb = est64 <= 128 ? 4 : (est64 <= 168 ? 3 : 2);
    }
    if (kind == kJitRegistersDD) {          // records in shared memory: 2 registers per value, ~90 besides
        const int estdd = 22 * g.R + 90;
        minb = estdd <= 128 ? 4 : (estdd <= 168 ? 3 : 2);
    }
    const int w = jit_warps(kind);
    minb = std::max(1, minb * kJitWarps / w);
    if (const char *ev = std::getenv("GRINS_JIT_MINB")) {
        const int m = std::atoi(ev);
        if (m >= 1 && m * w <= 64) minb = m;
    }
    return minb;
}

// Compiles the kernel for (g, kind) into e on device dev: from the block
// count of the register estimate, one block fewer while a register-record
// compile spills.  Wakes every thread waiting for an entry.
void jit_build_entry(JitEntry &e, const GrpTopo &g, int kind, int dev, int method)
{
    cudaSetDevice(dev);
    int minb = jit_minb(g, kind);
    const int warps = jit_warps(kind);
    JitBuild b;
    for (;;) {
        b = jit_compile(jit_main(g, kind, minb, warps, method));
        if (b.ok && kind != kJitShared && b.spill_bytes > 0 && minb > 1 && !std::getenv("GRINS_JIT_MINB") &&
            !jit_maxnreg(kind)) {
            cudaLibraryUnload(b.lib);
            --minb;
            continue;
        }
        break;
    }
    JitCache &c = jit_cache();
    {
        std::lock_guard<std::mutex> lock(c.mu);
        e.why = b.why;
        e.warps = warps;
        e.lib = b.lib;
        e.kern = b.kern;
        e.state.store(b.ok ? 1 : -1);
    }
    c.cv.notify_all();
}

enum JitMode { kLookup = 0, kCompileHere = 1, kCompileAsync = 2 };

// The cache entry for (g, kind), keyed by the source text of its first
// compile.  kLookup: null when absent; kCompileHere: compiles in this
// thread when absent and waits for a compile in flight; kCompileAsync:
// queues a background compile when absent and returns at once.
std::shared_ptr<JitEntry> jit_get(const GrpTopo &g, int kind, int mode, int method)
{
    const std::string key = jit_main(g, kind, jit_minb(g, kind), jit_warps(kind), method);
    JitCache &c = jit_cache();
    std::unique_lock<std::mutex> lock(c.mu);
    auto it = c.map.find(key);
    if (it == c.map.end()) {
        if (mode == kLookup) return nullptr;
        auto e = std::make_shared<JitEntry>();
        e->kind = kind;
        c.map.emplace(key, e);
        int dev = 0;
        cudaGetDevice(&dev);
        if (mode == kCompileHere) {
            lock.unlock();
            jit_build_entry(*e, g, kind, dev, method);
        } else {
            jit_pool_push([e, g, kind, dev, method] { jit_build_entry(*e, g, kind, dev, method); });
        }
        return e;
    }
    std::shared_ptr<JitEntry> e = it->second;
    if (mode == kCompileHere) c.cv.wait(lock, [&e] { return e->state.load() != 0; });
    return e;
}

bool jit_enabled(const GrpTopo &g, std::string *why)
{
    const char *ev = std::getenv("GRINS_JIT");
    if (ev && ev[0] == '0') { if (why) *why = "disabled by GRINS_JIT=0"; return false; }
    if (g.L <= 0 || g.R <= 0 || g.R > 12) { if (why) *why = "no lane-group layout"; return false; }
    return true;
}

}  // namespace

// The compiled kernel for layout g (compiling it on first use), or null
// with the reason in *why.  The pointer is an opaque handle for
// launch_grp_jit.
const void *grp_jit_kernel(const GrpTopo &g, int kind, std::string *why, int method)
{
    if (!jit_enabled(g, why)) return nullptr;
    if ((method & kJitMethodMask) != 0 && kind == kJitShared) {
        if (why) *why = "the shared-record kernel runs Dormand-Prince only";
        return nullptr;
    }
    std::shared_ptr<JitEntry> e = jit_get(g, kind, kCompileHere, method);
    if (e->state.load() != 1) { if (why) *why = e->why; return nullptr; }
    if (why)
        *why = e->kind == kJitRegisters64   ? "FP64, records in registers"
               : e->kind == kJitRegistersDD ? "double-float, records in registers"
               : e->kind == kJitRegisters   ? "records in registers"
                                            : "records in shared memory";
    return e.get();
}

// The compiled kernel for layout g if an earlier call compiled it; never
// compiles, loads or waits.
const void *grp_jit_lookup(const GrpTopo &g, int kind, int method)
{
    if (!jit_enabled(g, nullptr) || ((method & kJitMethodMask) != 0 && kind == kJitShared)) return nullptr;
    std::shared_ptr<JitEntry> e = jit_get(g, kind, kLookup, method);
    if (!e || e->state.load() != 1) return nullptr;
    return e.get();
}

// Starts (once) a background compile of the kernel for layout g and
// returns its state: 1 ready, 0 compiling, -1 failed or run-time compiles
// unavailable.
int grp_jit_prefetch(const GrpTopo &g, int kind, int method)
{
    if (!jit_enabled(g, nullptr) || ((method & kJitMethodMask) != 0 && kind == kJitShared)) return -1;
    return jit_get(g, kind, kCompileAsync, method)->state.load();
}

namespace {

// nvJitLink, opened with dlopen like NVRTC: the plan kernel is linked from
// separately compiled bodies.
struct JitLinkApi {
    bool ok = false;
    std::string why;
    decltype(&__nvJitLinkCreate_13_0) create = nullptr;
    decltype(&__nvJitLinkAddData_13_0) add_data = nullptr;
    decltype(&__nvJitLinkComplete_13_0) complete = nullptr;
    decltype(&__nvJitLinkGetLinkedCubinSize_13_0) cubin_size = nullptr;
    decltype(&__nvJitLinkGetLinkedCubin_13_0) cubin = nullptr;
    decltype(&__nvJitLinkGetErrorLogSize_13_0) err_size = nullptr;
    decltype(&__nvJitLinkGetErrorLog_13_0) err_log = nullptr;
    decltype(&__nvJitLinkDestroy_13_0) destroy = nullptr;
};

JitLinkApi &jitlink()
{
    static JitLinkApi api;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvJitLink.so.13", "libnvJitLink.so", "/usr/local/cuda/lib64/libnvJitLink.so.13",
                               "/usr/local/cuda/lib64/libnvJitLink.so"};
        void *h = nullptr;
        for (const char *n : names)
            if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) { api.why = "libnvJitLink not found"; return; }
        api.create = reinterpret_cast<decltype(api.create)>(dlsym(h, "nvJitLinkCreate"));
        api.add_data = reinterpret_cast<decltype(api.add_data)>(dlsym(h, "nvJitLinkAddData"));
        api.complete = reinterpret_cast<decltype(api.complete)>(dlsym(h, "nvJitLinkComplete"));
        api.cubin_size = reinterpret_cast<decltype(api.cubin_size)>(dlsym(h, "nvJitLinkGetLinkedCubinSize"));
        api.cubin = reinterpret_cast<decltype(api.cubin)>(dlsym(h, "nvJitLinkGetLinkedCubin"));
        api.err_size = reinterpret_cast<decltype(api.err_size)>(dlsym(h, "nvJitLinkGetErrorLogSize"));
        api.err_log = reinterpret_cast<decltype(api.err_log)>(dlsym(h, "nvJitLinkGetErrorLog"));
        api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "nvJitLinkDestroy"));
        api.ok = api.create && api.add_data && api.complete && api.cubin_size && api.cubin && api.err_size &&
                 api.err_log && api.destroy;
        if (!api.ok) api.why = "libnvJitLink lacks an expected symbol";
    });
    return api;
}

// NVRTC compile of relocatable device code (no load): the cubin, or empty
// with the reason in *why.
std::vector<char> rdc_compile(const std::string &src, int maxreg, std::string *why)
{
    NvrtcApi &api = nvrtc();
    if (!api.ok) { *why = api.why; return {}; }
    std::vector<const char *> hdr_src, hdr_name;
    for (int i = 0; i < kJitSourceCount; ++i) {
        hdr_src.push_back(kJitSources[i]);
        hdr_name.push_back(kJitSourceNames[i]);
    }
    hdr_src.push_back(kStdintStandIn);
    hdr_name.push_back("stdint.h");
    nvrtcProgram prog = nullptr;
    nvrtcResult r = api.create(&prog, src.c_str(), "grins_plan.cu", (int)hdr_src.size(), hdr_src.data(),
                               hdr_name.data());
    if (r != NVRTC_SUCCESS) { *why = std::string("nvrtcCreateProgram: ") + api.err(r); return {}; }
    const std::string reg = "--maxrregcount=" + std::to_string(maxreg);
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo", "-default-device",
                          "--relocatable-device-code=true", reg.c_str()};
    r = api.compile(prog, 6, opts);
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        api.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) api.log(prog, &log[0]);
        *why = std::string("nvrtcCompileProgram: ") + api.err(r) + "\n" + log;
        api.destroy(&prog);
        return {};
    }
    size_t n = 0;
    api.cubin_size(prog, &n);
    std::vector<char> cubin(n);
    api.cubin(prog, cubin.data());
    api.destroy(&prog);
    return cubin;
}

// One layout's integrator as a device function grins_body_<id> (FP32
// Dormand-Prince, no time series, no re-pass), compiled apart with the
// plan's register cap; cached per process by source and cap.
struct PlanBody {
    std::atomic<int> state{0};   // 0 compiling, 1 ready, -1 failed
    std::string why, name;
    std::vector<char> cubin;
};

struct PlanBodyCache {
    std::mutex mu;
    std::condition_variable cv;
    std::map<std::string, std::shared_ptr<PlanBody>> map;
};
PlanBodyCache &plan_body_cache()
{
    static PlanBodyCache *c = new PlanBodyCache();
    return *c;
}

std::string body_source(const GrpTopo &g, const std::string &name, bool cancel)
{
    std::string s = "#include \"common.cuh\"\n#include \"integrate_grp.cuh\"\nnamespace grins { namespace pkb {\n";
    s += layout_prelude(g, true);
    s += "#include \"integrate_rr_layout.inc\"\n} }\n";
    char buf[320];
    std::snprintf(buf, sizeof(buf),
                  "extern \"C\" __device__ __noinline__ void %s(const grins::IntegrateArgs &a, unsigned char *w)\n"
                  "{ grins::pkb::rr_body_at<%d, 4, %d, float, 0, false, false, %s>(a, w); }\n",
                  name.c_str(), g.R, g.L, cancel ? "true" : "false");
    return s + buf;
}

// The body for layout g under register cap maxreg: from the cache, or a
// compile queued on the host pool (the caller waits for it).
std::shared_ptr<PlanBody> plan_body(const GrpTopo &g, int maxreg, bool cancel)
{
    const std::string lay = layout_prelude(g, true) + "L=" + std::to_string(g.L) + " R=" + std::to_string(g.R);
    char id[64];
    std::snprintf(id, sizeof(id), "grins_body_%016zx_%d%s", std::hash<std::string>()(lay), maxreg, cancel ? "c" : "");
    const std::string src = body_source(g, id, cancel);
    const std::string key = src + "\nmaxreg " + std::to_string(maxreg);
    PlanBodyCache &c = plan_body_cache();
    std::lock_guard<std::mutex> lock(c.mu);
    auto it = c.map.find(key);
    if (it != c.map.end()) return it->second;
    auto b = std::make_shared<PlanBody>();
    b->name = id;
    c.map.emplace(key, b);
    jit_pool_push([b, src, maxreg] {
        std::string why;
        std::vector<char> cubin = rdc_compile(src, maxreg, &why);
        PlanBodyCache &cc = plan_body_cache();
        {
            std::lock_guard<std::mutex> l(cc.mu);
            b->cubin = std::move(cubin);
            b->why = why;
            b->state.store(b->cubin.empty() ? -1 : 1);
        }
        cc.cv.notify_all();
    });
    return b;
}

// The dispatcher: the job loop of plan_run with a switch over the bodies,
// which it declares and calls.
std::string plan_dispatch_source(const std::vector<std::shared_ptr<PlanBody>> &bodies, int warps, int minb)
{
    std::string s = "#include \"common.cuh\"\n#include \"integrate_plan.cuh\"\n";
    char buf[320];
    for (const auto &b : bodies) {
        std::snprintf(buf, sizeof(buf),
                      "extern \"C\" __device__ void %s(const grins::IntegrateArgs &a, unsigned char *w);\n",
                      b->name.c_str());
        s += buf;
    }
    std::snprintf(buf, sizeof(buf),
                  "extern \"C\" __global__ void __launch_bounds__(%d, %d) grins_plan_ct(const grins::PlanArgs p)\n{\n"
                  "    grins::plan_run(p, [](int body, const grins::IntegrateArgs &a, unsigned char *w) {\n"
                  "        switch (body) {\n", warps * kWarp, minb);
    s += buf;
    for (size_t i = 0; i < bodies.size(); ++i) {
        std::snprintf(buf, sizeof(buf), "        case %zu: %s(a, w); break;\n", i, bodies[i]->name.c_str());
        s += buf;
    }
    s += "        default: break;\n        }\n    });\n}\n";
    return s;
}

}  // namespace

// The plan kernel for n layouts with `minb` resident blocks of `warps`
// warps per SM (a register cap of 65536 / (32 warps minb) for every body):
// each distinct layout's body compiled apart (in parallel on the host pool,
// cached per layout and cap), a dispatcher compiled for this plan, linked
// with nvJitLink and loaded.  Cached by the dispatcher's source.
const void *grp_jit_plan_kernel(const GrpTopo *lay, int n, int warps, int minb, bool cancel, std::string *why)
{
    if (n < 1 || warps < 1 || minb < 1) { if (why) *why = "bad plan kernel request"; return nullptr; }
    for (int i = 0; i < n; ++i)
        if (!jit_enabled(lay[i], why)) return nullptr;
    JitLinkApi &lk = jitlink();
    if (!lk.ok) { if (why) *why = lk.why; return nullptr; }
    const int maxreg = std::min(255, 65536 / (warps * kWarp * minb) / 8 * 8);
    std::vector<std::shared_ptr<PlanBody>> bodies;
    for (int i = 0; i < n; ++i) bodies.push_back(plan_body(lay[i], maxreg, cancel));
    {
        PlanBodyCache &c = plan_body_cache();
        std::unique_lock<std::mutex> lock(c.mu);
        for (const auto &b : bodies) {
            c.cv.wait(lock, [&b] { return b->state.load() != 0; });
            if (b->state.load() != 1) { if (why) *why = "body compile: " + b->why; return nullptr; }
        }
    }
    const std::string key = plan_dispatch_source(bodies, warps, minb);
    JitCache &c = jit_cache();
    std::unique_lock<std::mutex> lock(c.mu);
    auto it = c.map.find(key);
    std::shared_ptr<JitEntry> e;
    if (it == c.map.end()) {
        e = std::make_shared<JitEntry>();
        e->kind = kJitRegisters;
        e->warps = warps;
        c.map.emplace(key, e);
        lock.unlock();
        std::string w;
        std::vector<char> disp = rdc_compile(key, maxreg, &w);
        std::vector<char> linked;
        if (!disp.empty()) {
            nvJitLinkHandle hl = nullptr;
            const std::string arch = "-arch=sm_103a";
            const char *lopts[] = {arch.c_str()};
            nvJitLinkResult lr = lk.create(&hl, 1, lopts);
            if (lr == NVJITLINK_SUCCESS) lr = lk.add_data(hl, NVJITLINK_INPUT_CUBIN, disp.data(), disp.size(), "dispatch");
            for (size_t i = 0; lr == NVJITLINK_SUCCESS && i < bodies.size(); ++i)
                lr = lk.add_data(hl, NVJITLINK_INPUT_CUBIN, bodies[i]->cubin.data(), bodies[i]->cubin.size(),
                                 bodies[i]->name.c_str());
            if (lr == NVJITLINK_SUCCESS) lr = lk.complete(hl);
            size_t sz = 0;
            if (lr == NVJITLINK_SUCCESS) lr = lk.cubin_size(hl, &sz);
            if (lr == NVJITLINK_SUCCESS) { linked.resize(sz); lr = lk.cubin(hl, linked.data()); }
            if (lr != NVJITLINK_SUCCESS) {
                size_t ln = 0;
                std::string log;
                if (hl && lk.err_size(hl, &ln) == NVJITLINK_SUCCESS && ln) { log.resize(ln); lk.err_log(hl, &log[0]); }
                w = "nvJitLink error " + std::to_string((int)lr) + ": " + log;
                linked.clear();
            }
            if (hl) lk.destroy(&hl);
        }
        cudaLibrary_t lib = nullptr;
        cudaKernel_t kern = nullptr;
        if (!linked.empty()) {
            cudaError_t ce = cudaLibraryLoadData(&lib, linked.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
            if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&kern, lib, "grins_plan_ct");
            if (ce != cudaSuccess) { w = std::string("loading the plan kernel: ") + cudaGetErrorString(ce); kern = nullptr; }
        }
        lock.lock();
        e->why = w;
        e->lib = lib;
        e->kern = kern;
        e->state.store(kern ? 1 : -1);
        c.cv.notify_all();
    } else {
        e = it->second;
        c.cv.wait(lock, [&e] { return e->state.load() != 0; });
    }
    if (e->state.load() != 1) { if (why) *why = e->why; return nullptr; }
    if (why) why->clear();
    return e.get();
}

cudaError_t launch_plan_ct(const void *handle, const PlanArgs &p, cudaStream_t st, int num_sms, int smem_limit)
{
    const JitEntry *je = static_cast<const JitEntry *>(handle);
    if (je->state.load() != 1) return cudaErrorInvalidValue;
    const int smem = je->warps * p.region_bytes;
    if (smem > smem_limit) return cudaErrorInvalidConfiguration;
    const void *kern = reinterpret_cast<const void *>(je->kern);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, je->warps * kWarp, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    PlanArgs q = p;
    void *args[] = {&q};
    err = cudaLaunchKernel(kern, dim3((unsigned)(num_sms * per_sm)), dim3(je->warps * kWarp), args, (size_t)smem, st);
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

cudaError_t launch_grp_jit(const void *handle, const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    const JitEntry *je = static_cast<const JitEntry *>(handle);
    if (je->state.load() != 1) return cudaErrorInvalidValue;
    IntegrateArgs b = a;
    const int W = je->warps;
    int smem = 0;
    if (je->kind != kJitShared) {
        smem = je->kind == kJitRegisters     ? W * rr_warp_bytes(b.grp.R, 1, 4)
               : je->kind == kJitRegistersDD ? W * rr_dd_warp_bytes(b.grp.R, b.grp.P)
                                             : W * rr_warp_bytes(b.grp.R, 6, 8);
    } else {
        const int ndom = grp_domains(b.grp.L);
        GrpLayout LY{b.grp.L, b.grp.R, b.grp.P, b.slots};
        while (kJitWarps * LY.warp_bytes() > b.smem_limit && LY.S > ndom) LY.S = (b.slots -= ndom);
        smem = kJitWarps * LY.warp_bytes();
    }
    if (smem > b.smem_limit) return cudaErrorInvalidConfiguration;
    const void *kern = reinterpret_cast<const void *>(je->kern);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * kWarp, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int groups = kWarp / b.grp.L;
    const long long work_warps = (b.n_sets * b.n_ics + groups - 1) / groups + 1;
    long long blocks = (long long)num_sms * per_sm;
    const long long need = (work_warps + W - 1) / W;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    void *args[] = {&b};
    err = cudaLaunchKernel(kern, dim3((unsigned)blocks), dim3(W * kWarp), args, (size_t)smem, st);
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

}  // namespace grins
