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
    std::snprintf(buf, sizeof(buf), "constexpr int kGrpCtRows = %d;\n", g.R);
    s += buf;
    s += "template <int r> struct GrpRowCt { static constexpr int off = 0, deg = 0, link = -1; };\n";
    for (int r = 0; r < g.R; ++r) {
        std::snprintf(buf, sizeof(buf),
                      "template <> struct GrpRowCt<%d> { static constexpr int off = %d, deg = %d, link = %d; };\n",
                      r, g.row_off[r], g.row_deg[r], kind == kJitShared ? -1 : g.link_to[r]);
        s += buf;
    }
    if (kind == kJitRegisters || kind == kJitRegisters64) {
        s += "}\n#include \"integrate_rr.cuh\"\n";
        char bounds[64];
        if (const int mr = jit_maxnreg(kind)) std::snprintf(bounds, sizeof(bounds), "__maxnreg__(%d)", mr);
        else std::snprintf(bounds, sizeof(bounds), "__launch_bounds__(%d, %d)", warps * kWarp, minb);
        std::snprintf(buf, sizeof(buf),
                      "extern \"C\" __global__ void %s grins_grp_ct(const grins::IntegrateArgs a)\n"
                      "{\n    grins::rr_body<%d, %d, %d, %s, %d>(a);\n}\n",
                      bounds, g.R, warps, g.L, kind == kJitRegisters64 ? "double" : "float", method);
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

JitBuild jit_compile(const std::string &src)
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
    if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&b.kern, b.lib, "grins_grp_ct");
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
    if (method != 0 && kind == kJitShared) {
        if (why) *why = "the shared-record kernel runs Dormand-Prince only";
        return nullptr;
    }
    std::shared_ptr<JitEntry> e = jit_get(g, kind, kCompileHere, method);
    if (e->state.load() != 1) { if (why) *why = e->why; return nullptr; }
    if (why)
        *why = e->kind == kJitRegisters64 ? "FP64, records in registers"
                                          : (e->kind == kJitRegisters ? "records in registers" : "records in shared memory");
    return e.get();
}

// The compiled kernel for layout g if an earlier call compiled it; never
// compiles, loads or waits.
const void *grp_jit_lookup(const GrpTopo &g, int kind, int method)
{
    if (!jit_enabled(g, nullptr) || (method != 0 && kind == kJitShared)) return nullptr;
    std::shared_ptr<JitEntry> e = jit_get(g, kind, kLookup, method);
    if (!e || e->state.load() != 1) return nullptr;
    return e.get();
}

// Starts (once) a background compile of the kernel for layout g and
// returns its state: 1 ready, 0 compiling, -1 failed or run-time compiles
// unavailable.
int grp_jit_prefetch(const GrpTopo &g, int kind, int method)
{
    if (!jit_enabled(g, nullptr) || (method != 0 && kind == kJitShared)) return -1;
    return jit_get(g, kind, kCompileAsync, method)->state.load();
}

cudaError_t launch_grp_jit(const void *handle, const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    const JitEntry *je = static_cast<const JitEntry *>(handle);
    if (je->state.load() != 1) return cudaErrorInvalidValue;
    IntegrateArgs b = a;
    const int W = je->warps;
    int smem = 0;
    if (je->kind == kJitRegisters || je->kind == kJitRegisters64) {
        smem = je->kind == kJitRegisters ? W * rr_warp_bytes(b.grp.R, 1, 4) : W * rr_warp_bytes(b.grp.R, 6, 8);
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
