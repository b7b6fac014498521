// C ABI of the GB300 BCMG library: handle life cycle, argument checks,
// stream ordering, CUDA-graph replay of the V-cycle, and error reporting.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "bcmg_internal.cuh"

namespace bcmg {

namespace {
thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}
}  // namespace

void check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        std::string m = std::string(what) + ": " + cudaGetErrorString(e);
        throw Error{e == cudaErrorMemoryAllocation ? BCMG_ENOMEM : BCMG_ECUDA, m};
    }
}

// Device memory of a handle.  Arrays up to kSmallAlloc bytes are carved from
// kChunk-byte chunks that are zero-filled once when taken; larger arrays get
// their own block, zero-filled only when the caller needs zeros.  Blocks
// come from a process-wide cache keyed by (device, size) before the
// device's stream-ordered pool: the blocks of a destroyed handle, or of a
// finished set-up's scratch, enter the cache only after every stream that
// used them has been synchronised, so any stream may take them, and
// repeated creations of the same hierarchy (a benchmark loop, a batch of
// equal problems) need no driver call at all.  A miss returns the device's
// cached blocks to the pool first (stream-ordered frees), so that a mix of
// sizes reuses the pool's memory instead of growing it around blocks that
// no one takes.  At most kCacheMax bytes are cached; when the pool cannot
// allocate, the cache goes back to the driver and the allocation is retried
// once.
constexpr size_t kChunk = 4u << 20;
constexpr size_t kSmallAlloc = 256u << 10;
constexpr size_t kCacheMax = 4ull << 30;

std::mutex g_cache_mu;
std::multimap<std::pair<int, size_t>, void *> g_cache;
size_t g_cache_bytes = 0;

// a block of exactly this size, else nullptr after the device's cached
// blocks went back to the pool (freed on st, where the caller allocates next)
void *cache_take(int dev, size_t bytes, cudaStream_t st) {
    std::vector<void *> back;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_cache.find({dev, bytes});
        if (it != g_cache.end()) {
            void *p = it->second;
            g_cache.erase(it);
            g_cache_bytes -= bytes;
            return p;
        }
        for (auto jt = g_cache.lower_bound({dev, 0}); jt != g_cache.end() && jt->first.first == dev;) {
            back.push_back(jt->second);
            g_cache_bytes -= jt->first.second;
            jt = g_cache.erase(jt);
        }
    }
    for (void *p : back) cudaFreeAsync(p, st);
    return nullptr;
}

// p is idle on every stream; past the cap it is freed on st instead
void cache_put(int dev, size_t bytes, void *p, cudaStream_t st) {
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        if (g_cache_bytes + bytes <= kCacheMax) {
            g_cache.emplace(std::make_pair(dev, bytes), p);
            g_cache_bytes += bytes;
            return;
        }
    }
    cudaFreeAsync(p, st);
}

void cache_drain() {
    std::multimap<std::pair<int, size_t>, void *> all;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        all.swap(g_cache);
        g_cache_bytes = 0;
    }
    int cur = 0;
    (void)cudaGetDevice(&cur);
    for (auto &kv : all) {
        (void)cudaSetDevice(kv.first.first);
        (void)cudaFree(kv.second);
    }
    (void)cudaSetDevice(cur);
}

bool in_workspace(const Handle &H, const void *p) {
    return H.ws_base && (const char *)p >= H.ws_base && (const char *)p < H.ws_base + H.ws_cap;
}

// Allocation-failure injection (bcmg_debug_fail_allocation): when the
// countdown reaches zero the device allocation fails as if the pool were
// exhausted.  Host-side only: no GPU fault is involved.
std::atomic<int64_t> g_fail_countdown{0};
// device blocks (and bytes) held by live handles, outside the cache
std::atomic<int64_t> g_live_blocks{0}, g_live_bytes{0};

void release_block(Handle &H, void *p, size_t bytes) {
    if (in_workspace(H, p)) return;
    g_live_blocks.fetch_sub(1);
    g_live_bytes.fetch_sub((int64_t)bytes);
    cache_put(H.dev, bytes, p, H.st);
}

bool injected_failure() {
    int64_t c = g_fail_countdown.load();
    while (c > 0) {
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}

void *raw_alloc(Handle &H, size_t bytes, bool temp) {
    if (injected_failure())
        throw Error{BCMG_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected)"};
    void *p = nullptr;
    if (H.ws_base) {
        // the caller's workspace: bump allocation, 256-byte aligned
        const size_t off = (H.ws_used + 255) & ~(size_t)255;
        if (off + bytes > H.ws_cap)
            throw Error{BCMG_ENOMEM, "workspace too small: " + std::to_string(H.ws_cap) + " bytes given, more than " +
                                         std::to_string(off + bytes) + " needed"};
        p = H.ws_base + off;
        H.ws_used = off + bytes;
        H.alloc_total = (int64_t)H.ws_used;
        (temp ? H.temps : H.allocs).push_back({p, bytes});
        if (!temp) H.dev_bytes += (int64_t)bytes;
        return p;
    }
    p = cache_take(H.dev, bytes, H.st);
    if (!p) {
        cudaError_t e = cudaMallocAsync(&p, bytes, H.st);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            cache_drain();
            e = cudaMallocAsync(&p, bytes, H.st);
        }
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            throw Error{BCMG_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
        }
    }
    (temp ? H.temps : H.allocs).push_back({p, bytes});
    if (!temp) H.dev_bytes += (int64_t)bytes;
    H.alloc_total += (int64_t)bytes;
    g_live_blocks.fetch_add(1);
    g_live_bytes.fetch_add((int64_t)bytes);
    return p;
}

void *dalloc(Handle &H, size_t bytes, bool temp, bool zero) {
    bytes = (std::max<size_t>(bytes, 8) + 255) & ~(size_t)255;
    if (bytes <= kSmallAlloc) {
        Arena &A = temp ? H.arena_temp : H.arena_perm;
        if (!A.base || A.used + bytes > A.cap) {
            A.base = (char *)raw_alloc(H, kChunk, temp);
            A.used = 0;
            A.cap = kChunk;
            check_cuda(cudaMemsetAsync(A.base, 0, kChunk, H.st), "cudaMemsetAsync");
        }
        void *p = A.base + A.used;
        A.used += bytes;
        return p;
    }
    void *p = raw_alloc(H, bytes, temp);
    if (zero) check_cuda(cudaMemsetAsync(p, 0, bytes, H.st), "cudaMemsetAsync");
    return p;
}

void count_launch(Handle &H) {
    if (H.capturing) H.captured++;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}

int64_t launches_total() { return g_launches.load(); }

void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int report(int code, const std::string &msg) {
    if (code == BCMG_OK) g_last_error.clear();
    else g_last_error = msg;
    return code;
}

void profile_mark(Handle &H, const Level &L) {
    if (!H.o.profile || H.L.empty() || &L != &H.L[0]) return;
    if (H.pev_next >= (int)H.pev.size()) return;
    check_cuda(cudaEventRecordWithFlags(H.pev[H.pev_next], H.st, H.capturing ? cudaEventRecordExternal : 0),
               "profile event");
    H.pev_next++;
}

namespace {

// H's streams are synchronised (creation's closing sync, or destroy)
void free_temps(Handle &H) {
    for (auto &pb : H.temps) release_block(H, pb.first, pb.second);
    H.temps.clear();
    H.arena_temp = Arena{};
}

// once per device (an attribute of the device's default pool)
std::mutex g_pool_mu;
std::vector<int> g_pool_devs;

void keep_pool_memory() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (std::find(g_pool_devs.begin(), g_pool_devs.end(), dev) != g_pool_devs.end()) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t thr = UINT64_MAX;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr) == cudaSuccess) g_pool_devs.push_back(dev);
}

// Small pinned host blocks (norms, solve state) come from a process-wide
// pool that is never returned to the driver: cudaFreeHost waits for the
// whole device, which would make every handle's destroy wait for the work
// of all other handles in flight.
constexpr size_t kPinBlock = 256;
std::mutex g_pin_mu;
std::vector<void *> g_pin_free;

void *pinned_get() {
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (!g_pin_free.empty()) {
            void *p = g_pin_free.back();
            g_pin_free.pop_back();
            return p;
        }
    }
    void *p = nullptr;
    check_cuda(cudaMallocHost(&p, kPinBlock), "cudaMallocHost");
    return p;
}

void pinned_put(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

// Streams with two events each ("lanes") come from a process-wide pool per
// device: a handle's own stream (with its enter and leave events) for its
// lifetime, and the side stream of a creation (with its fork and join
// events) while the hierarchy is built.  A lane goes back idle (its stream
// synchronised), so that handles created and destroyed at a high rate make
// no stream or event calls, which take driver locks that concurrent
// creations would contend for.  A recorded event may be reused at once: a
// stream that waits on it waits for the record made before its wait call.
struct SideLane {
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
std::mutex g_side_mu;
std::vector<std::pair<int, SideLane>> g_side_free;

SideLane side_get(int dev) {
    {
        std::lock_guard<std::mutex> lk(g_side_mu);
        for (size_t i = 0; i < g_side_free.size(); ++i)
            if (g_side_free[i].first == dev) {
                SideLane s = g_side_free[i].second;
                g_side_free.erase(g_side_free.begin() + (int64_t)i);
                return s;
            }
    }
    SideLane s;
    check_cuda(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking), "cudaStreamCreate");
    check_cuda(cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming), "cudaEventCreate");
    check_cuda(cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming), "cudaEventCreate");
    return s;
}

void lane_put(int dev, SideLane s) {
    std::lock_guard<std::mutex> lk(g_side_mu);
    g_side_free.push_back({dev, s});
}

// the lane is idle (its stream synchronised)
void side_put(int dev, Handle &H) {
    if (!H.st2) return;
    SideLane s;
    s.st = H.st2;
    s.fork = H.ev_fork;
    s.join = H.ev_join;
    H.st2 = nullptr;
    H.ev_fork = H.ev_join = nullptr;
    std::lock_guard<std::mutex> lk(g_side_mu);
    g_side_free.push_back({dev, s});
}

void destroy(Handle *H) {
    if (!H) return;
    if (H->st2) cudaStreamSynchronize(H->st2);
    if (H->st) cudaStreamSynchronize(H->st);
    if (H->vgraph) cudaGraphExecDestroy(H->vgraph);
    if (H->ngraph) cudaGraphExecDestroy(H->ngraph);
    if (H->sgraph) cudaGraphExecDestroy(H->sgraph);
    pinned_put(H->shost);
    if (H->st) {
        free_temps(*H);
        for (auto &pb : H->allocs) release_block(*H, pb.first, pb.second);
        H->allocs.clear();
        cudaStreamSynchronize(H->st);
    }
    pinned_put(H->nhost);
    pinned_put(H->sing_host);
    for (cudaEvent_t e : H->pev) cudaEventDestroy(e);
    side_put(H->dev, *H);  // synchronised above
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (H->st && cudaStreamIsCapturing(H->st, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusInvalidated;
    if (H->st && H->ev_in && H->ev_out && cap == cudaStreamCaptureStatusNone) {  // synchronised above
        lane_put(H->dev, SideLane{H->st, H->ev_in, H->ev_out});
    } else {
        if (H->ev_in) cudaEventDestroy(H->ev_in);
        if (H->ev_out) cudaEventDestroy(H->ev_out);
        if (H->st) cudaStreamDestroy(H->st);
    }
    H->magic = 0;
    delete H;
}

// order the library stream after the caller's stream, and back
void enter(Handle &H) {
    check_cuda(cudaEventRecord(H.ev_in, H.user), "cudaEventRecord(in)");
    check_cuda(cudaStreamWaitEvent(H.st, H.ev_in, 0), "cudaStreamWaitEvent(in)");
}

void leave(Handle &H) {
    check_cuda(cudaEventRecord(H.ev_out, H.st), "cudaEventRecord(out)");
    check_cuda(cudaStreamWaitEvent(H.user, H.ev_out, 0), "cudaStreamWaitEvent(out)");
}

// Capture fn() on the library stream into an executable graph.
template <class Fn>
cudaGraphExec_t capture(Handle &H, int64_t *kernels, Fn fn) {
    cudaGraph_t g = nullptr;
    check_cuda(cudaStreamBeginCapture(H.st, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    H.capturing = true;
    H.captured = 0;
    H.pev_next = 0;
    try {
        fn();
    } catch (...) {
        H.capturing = false;
        cudaStreamEndCapture(H.st, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    H.capturing = false;
    H.pev_pairs = H.pev_next / 2;
    check_cuda(cudaStreamEndCapture(H.st, &g), "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    check_cuda(e, "cudaGraphInstantiate");
    *kernels = H.captured;
    return ex;
}

// one cycle on the working copy: a V-cycle (FP64), or one refinement step
// (FP64 residual, FP32 V-cycle on the correction, FP64 update)
void cycle_body(Handle &H) {
    if (H.o.precision == BCMG_PREC_MIXED) {
        Level &L = H.L[0];
        residual<double>(H, L, H.u0, L.F, L.r);
        mixed_step_enqueue(H, H.u0);
    } else {
        vcycle_enqueue(H, 0, H.u0);
    }
}

void run_vcycle(Handle &H) {
    if (H.o.use_graph) {
        if (!H.vgraph) H.vgraph = capture(H, &H.vgraph_kernels, [&] { cycle_body(H); });
        check_cuda(cudaGraphLaunch(H.vgraph, H.st), "cudaGraphLaunch(vcycle)");
        g_launches.fetch_add(H.vgraph_kernels, std::memory_order_relaxed);
    } else {
        cycle_body(H);
    }
}

void enqueue_norms(Handle &H) {
    residual_norms(H, H.u0, H.nout);
}

// The norms after a cycle may take the residual's after-smoothing form: an
// FP64 cycle ends with a red-black smoothing step of the finest level (a
// refinement step ends with its correction instead)
bool norms_after_rb(const Handle &H) {
    return H.o.precision == BCMG_PREC_FP64 && H.o.ordering == BCMG_ORDER_RB && H.o.nu2 > 0 && H.L.size() > 1;
}

// add the device time of the profiled sweeps of the last completed cycle
void profile_collect(Handle &H) {
    if (!H.o.profile) return;
    for (int p = 0; p < H.pev_pairs; ++p) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, H.pev[2 * p], H.pev[2 * p + 1]) == cudaSuccess) {
            H.prof_ms += ms;
            H.prof_n++;
        } else {
            (void)cudaGetLastError();
        }
    }
}

// cycle + residual norms of the result (one graph).  In mixed precision the
// finest residual r left by the previous norms is the refinement's input.
void solve_body(Handle &H) {
    if (H.o.precision == BCMG_PREC_MIXED) mixed_step_enqueue(H, H.u0);
    else vcycle_enqueue(H, 0, H.u0);
    residual_norms(H, H.u0, H.nout, 0, 0, norms_after_rb(H));
}

void run_vcycle_norms(Handle &H) {
    if (!H.o.use_graph) H.pev_next = 0;
    if (H.o.use_graph) {
        if (!H.ngraph) H.ngraph = capture(H, &H.ngraph_kernels, [&] { solve_body(H); });
        check_cuda(cudaGraphLaunch(H.ngraph, H.st), "cudaGraphLaunch(vcycle+norms)");
        g_launches.fetch_add(H.ngraph_kernels, std::memory_order_relaxed);
    } else {
        solve_body(H);
        H.pev_pairs = H.pev_next / 2;
    }
}

// The whole solve as one graph: residual norms of the start and the solve's
// start (r0, first condition), then a WHILE conditional node whose body is
// one cycle, its residual norms and the convergence check (which sets the
// condition).  No host round trip per
// cycle.  Built once per handle; on any failure the handle falls back to the
// host-driven loop of cycle graphs.
cudaGraphExec_t build_solve_graph(Handle &H) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool capturing = false;
    try {
        check_cuda(cudaGraphCreate(&g, 0), "cudaGraphCreate");
        cudaGraphConditionalHandle cond;
        check_cuda(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault),
                   "cudaGraphConditionalHandleCreate");
        check_cuda(cudaStreamBeginCaptureToGraph(H.st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                   "capture solve prefix");
        capturing = true;
        H.capturing = true;
        H.captured = 0;
        residual_norms(H, H.u0, H.nout, 1, (unsigned long long)cond);
        H.sgraph_prefix = H.captured;
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        check_cuda(cudaStreamGetCaptureInfo(H.st, &cs, nullptr, nullptr, &deps, nullptr, &nd), "capture info");
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = cond;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t cn;
        check_cuda(cudaGraphAddNode(&cn, g, deps, nullptr, nd, &p), "add WHILE node");
        check_cuda(cudaStreamUpdateCaptureDependencies(H.st, &cn, nullptr, 1, cudaStreamSetCaptureDependencies),
                   "capture dependencies");
        capturing = false;
        check_cuda(cudaStreamEndCapture(H.st, &g), "end capture solve prefix");
        cudaGraph_t body = p.conditional.phGraph_out[0];
        check_cuda(cudaStreamBeginCaptureToGraph(H.st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                   "capture solve body");
        capturing = true;
        H.captured = 0;
        if (H.o.precision == BCMG_PREC_MIXED) mixed_step_enqueue(H, H.u0);
        else vcycle_enqueue(H, 0, H.u0);
        residual_norms(H, H.u0, H.nout, 2, (unsigned long long)cond, norms_after_rb(H));
        H.sgraph_body = H.captured;
        capturing = false;
        check_cuda(cudaStreamEndCapture(H.st, &body), "end capture solve body");
        H.capturing = false;
        check_cuda(cudaGraphInstantiate(&ex, g, 0), "instantiate solve graph");
        cudaGraphDestroy(g);
        return ex;
    } catch (const Error &) {
        H.capturing = false;
        if (capturing) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(H.st, &junk);
        }
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        H.sgraph_failed = true;
        return nullptr;
    }
}

void fetch_norms(Handle &H, double out[4]) {
    check_cuda(cudaMemcpyAsync(H.nhost, H.nout, 4 * sizeof(double), cudaMemcpyDeviceToHost, H.st), "norms D2H");
    check_cuda(cudaStreamSynchronize(H.st), "norms sync");
    for (int i = 0; i < 4; ++i) out[i] = H.nhost[i];
}

Handle *checked(bcmg_handle h) {
    if (!h) throw Error{BCMG_EINVAL, "null handle"};
    Handle *H = reinterpret_cast<Handle *>(h);
    if (H->magic != kHandleMagic) throw Error{BCMG_EINVAL, "not a live handle"};
    return H;
}

Level &level_of(Handle &H, int l) {
    if (l < 0 || l >= (int)H.L.size()) throw Error{BCMG_EINVAL, "level out of range"};
    return H.L[l];
}

template <class Fn>
int guarded(Fn fn) {
    try {
        fn();
        g_last_error.clear();
        return BCMG_OK;
    } catch (const Error &e) {
        return fail(e.code, e.msg);
    } catch (const std::bad_alloc &) {
        return fail(BCMG_ENOMEM, "host allocation failed");
    } catch (...) {
        return fail(BCMG_ECUDA, "unexpected exception");
    }
}

// The solve state in and out without the copy engines: in as a launch
// parameter, out by a store into the pinned block through its device alias.
// A small copy is queued behind the large transfers other streams have in
// flight (a caller's next inputs, a previous result on its way back), so a
// copy here would hold the solve until they finished.
__global__ void k_state_put(SolveState *d, SolveState s) {
    if (threadIdx.x == 0) *d = s;
}

__global__ void k_state_get(SolveState *h, const SolveState *d) {
    if (threadIdx.x == 0) *h = *d;
}

// Enqueue a whole device-driven solve on the handle's stream (no host wait):
// copy u in, the solve graph, the state back, u out.  False if this handle
// solves with the host loop instead (profiling, graphs off, or no graph).
bool solve_enqueue(Handle &H, double *u_dev, double rtol, int max_cycles) {
    if (!H.o.use_graph || H.o.profile) return false;
    if (!H.sgraph && !H.sgraph_failed) H.sgraph = build_solve_graph(H);
    if (!H.sgraph) return false;
    enter(H);
    copy_active(H, u_dev, H.u0, true);
    H.shost->rtol = rtol;
    H.shost->max_cycles = max_cycles;
    if (H.shost_dev) {
        k_state_put<<<1, 32, 0, H.st>>>(H.sdev, *H.shost);
        check_cuda(cudaGetLastError(), "k_state_put");
    } else {
        check_cuda(cudaMemcpyAsync(H.sdev, H.shost, sizeof(SolveState), cudaMemcpyHostToDevice, H.st),
                   "solve state H2D");
    }
    check_cuda(cudaGraphLaunch(H.sgraph, H.st), "cudaGraphLaunch(solve)");
    if (H.shost_dev) {
        k_state_get<<<1, 32, 0, H.st>>>(H.shost_dev, H.sdev);
        check_cuda(cudaGetLastError(), "k_state_get");
        add_launches(2);
    } else {
        check_cuda(cudaMemcpyAsync(H.shost, H.sdev, sizeof(SolveState), cudaMemcpyDeviceToHost, H.st),
                   "solve state D2H");
    }
    copy_active(H, H.u0, u_dev, false);
    leave(H);
    return true;
}

// wait for an enqueued solve and read its state
int solve_finish(Handle &H, double rtol, int *cycles, double *rel) {
    check_cuda(cudaStreamSynchronize(H.st), "solve sync");
    const SolveState &s = *H.shost;
    *cycles = s.cycles;
    *rel = s.rel;
    add_launches(H.sgraph_prefix + H.sgraph_body * (int64_t)s.cycles);
    int status = s.status;
    if (status == BCMG_OK && s.r0 > 0.0 && s.rel > rtol) status = BCMG_ENOCONV;
    return status;
}

// host-driven loop over captured cycle graphs (or plain launches), reading
// the norms after every cycle
int solve_host_loop(Handle &H, double *u_dev, double rtol, int max_cycles, int *cycles, double *rel_out) {
    int status = BCMG_OK;
    enter(H);
    copy_active(H, u_dev, H.u0, true);
    enqueue_norms(H);
    double nr[4];
    fetch_norms(H, nr);
    // sqrt(a^2 + b^2) rounded step by step, as the device's solve control
    // does (the library's host code is built without FMA contraction)
    const double r0 = std::sqrt(nr[0] * nr[0] + nr[1] * nr[1]);
    double rel = (r0 > 0.0) ? 1.0 : 0.0;
    int c = 0;
    if (!std::isfinite(r0)) status = BCMG_ENONFINITE;
    while (status == BCMG_OK && r0 > 0.0 && c < max_cycles) {
        run_vcycle_norms(H);
        fetch_norms(H, nr);
        profile_collect(H);
        ++c;
        const double rn = std::sqrt(nr[0] * nr[0] + nr[1] * nr[1]);
        rel = rn / r0;
        if (!std::isfinite(rn)) status = BCMG_ENONFINITE;
        else if (rel <= rtol) break;
    }
    if (status == BCMG_OK && r0 > 0.0 && rel > rtol) status = BCMG_ENOCONV;
    copy_active(H, H.u0, u_dev, false);
    leave(H);
    *cycles = c;
    *rel_out = rel;
    return status;
}

int solve_status(int status) {
    if (status == BCMG_ENOCONV) return fail(status, "max_cycles reached before rtol");
    if (status == BCMG_ENONFINITE) return fail(status, "non-finite residual");
    g_last_error.clear();
    return BCMG_OK;
}

// The stage operators take the caller's arrays in the dense layout; the
// kernels work on the parity-split one, so the arrays go through the
// handle's stage scratch (allocated on the first stage call, three arrays
// of the finest level's split length, from the library's allocator even
// when the hierarchy lives in a caller workspace).
double *stage_buf(Handle &H, int k) {
    if (!H.stage[k]) {
        char *ws = H.ws_base;
        H.ws_base = nullptr;
        try {
            H.stage[k] = (double *)dalloc(H, sizeof(double) * split_len(H.L[0].nn), false, false);
        } catch (...) {
            H.ws_base = ws;
            throw;
        }
        H.ws_base = ws;
    }
    return H.stage[k];
}

// host memory (pageable or page-locked), as opposed to device or managed
bool is_host_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

// the handles of a batch call: live, distinct, each with its u
std::vector<Handle *> batch_handles(bcmg_handle *handles, double **u_devs, int n) {
    std::vector<Handle *> hs(n);
    for (int i = 0; i < n; ++i) {
        hs[i] = checked(handles[i]);
        if (!u_devs[i]) throw Error{BCMG_EINVAL, "null u in batch"};
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) throw Error{BCMG_EINVAL, "a handle appears twice in the batch"};
    }
    return hs;
}

// An eligible batch through the batched kernels (batch.cu), on the first
// handle's stream.  It waits once for every distinct caller stream (each
// handle's earlier work is ordered before its caller's stream), copies every
// u in with one launch and out with one, and is synchronised before the
// return, so each caller stream finds its u written and each handle's stream
// its arrays idle.  fixed: exactly max_cycles cycles (batched V-cycles).
void batched_run(const std::vector<Handle *> &hs, double **u_devs, double rtol, int max_cycles, bool fixed,
                 int *cyc, double *rel, int *st) {
    cudaStream_t bst = hs[0]->st;
    std::vector<cudaStream_t> users;
    for (Handle *H : hs) {
        if (std::find(users.begin(), users.end(), H->user) != users.end()) continue;
        users.push_back(H->user);
        check_cuda(cudaEventRecord(H->ev_in, H->user), "batch fork");
        check_cuda(cudaStreamWaitEvent(bst, H->ev_in, 0), "batch fork wait");
    }
    batch_copy_active(hs, u_devs, bst, true);
    add_launches(batch_solve(hs, bst, rtol, max_cycles, cyc, rel, st, fixed));
    batch_copy_active(hs, u_devs, bst, false);
    check_cuda(cudaStreamSynchronize(bst), "batch sync");
}

}  // namespace
}  // namespace bcmg

using namespace bcmg;

extern "C" {

void bcmg_default_opts(bcmg_opts *o) {
    if (!o) return;
    o->nu1 = 2;
    o->nu2 = 1;
    o->dtau_mode = BCMG_DTAU_EXP;
    o->dtau_const = 1.75;
    o->ext_sweeps = 4;
    o->min_coarse = 8;
    o->max_levels = 24;
    o->use_graph = 1;
    o->profile = 0;
    o->precision = BCMG_PREC_FP64;
    o->bc = BCMG_BC_DIRICHLET;
    o->reaction = 0.0;
    o->cycle = BCMG_CYCLE_V;
    o->ordering = BCMG_ORDER_RB;
    o->tg_inner = 30;
}

int bcmg_create_grid_hierarchy(int dim, int64_t N, const double *phi_dev, const double *f_dev,
                               const bcmg_opts *opts, void *stream, bcmg_handle *out) {
    return bcmg_create_grid_hierarchy_ex(dim, N, -1.0, N > 0 ? 2.0 / (double)N : 0.0, phi_dev, f_dev, opts,
                                         nullptr, 0, stream, out);
}

int bcmg_create_grid_hierarchy_ex(int dim, int64_t N, double lo, double h, const double *phi_dev,
                                  const double *f_dev, const bcmg_opts *opts, void *workspace, size_t ws_bytes,
                                  void *stream, bcmg_handle *out) {
    if (!out) return fail(BCMG_EINVAL, "out is null");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(BCMG_EINVAL, "dim must be 2 or 3");
    if (N < 4 || N > 65534) return fail(BCMG_EINVAL, "N must be in [4, 65534]");
    double nn_d = std::pow((double)(N + 1), dim);
    if (nn_d >= 4294967295.0) return fail(BCMG_EINVAL, "grid has 2^32 nodes or more");
    if (!phi_dev) return fail(BCMG_EINVAL, "phi is null");
    if (!std::isfinite(lo) || !(h > 0.0) || !std::isfinite(h) || !std::isfinite(lo + (double)N * h))
        return fail(BCMG_EINVAL, "lo must be finite and h positive and finite");
    if (workspace && (ws_bytes == 0 || ((uintptr_t)workspace & 255u) != 0))
        return fail(BCMG_EINVAL, "workspace must be 256-byte aligned with ws_bytes > 0");
    Handle *H = nullptr;
    int rc = guarded([&] {
        H = new Handle();
        H->d = dim;
        H->N = N;
        H->lo = lo;
        H->h0 = h;
        H->ws_base = (char *)workspace;
        H->ws_cap = workspace ? ws_bytes : 0;
        if (opts) H->o = *opts;
        else bcmg_default_opts(&H->o);
        if (H->o.nu1 < 0 || H->o.nu2 < 0 || H->o.ext_sweeps < 1 || H->o.min_coarse < 2 ||
            H->o.max_levels < 1 || H->o.dtau_mode < 0 || H->o.dtau_mode > 2 ||
            (H->o.precision != BCMG_PREC_FP64 && H->o.precision != BCMG_PREC_MIXED) ||
            (H->o.bc != BCMG_BC_DIRICHLET && H->o.bc != BCMG_BC_NEUMANN) ||
            !(H->o.reaction >= 0.0 && H->o.reaction < 1e300) ||
            (H->o.cycle != BCMG_CYCLE_V && H->o.cycle != BCMG_CYCLE_W && H->o.cycle != BCMG_CYCLE_TG) ||
            (H->o.cycle == BCMG_CYCLE_TG && (H->o.tg_inner < 1 || H->o.tg_inner > 10000)) ||
            (H->o.ordering != BCMG_ORDER_RB && H->o.ordering != BCMG_ORDER_LEX) || H->o.use_graph < 0 ||
            H->o.use_graph > 2)
            throw Error{BCMG_EINVAL, "invalid options"};
        H->user = (cudaStream_t)stream;
        check_cuda(cudaGetDevice(&H->dev), "cudaGetDevice");
        keep_pool_memory();
        {
            SideLane ml = side_get(H->dev);
            H->st = ml.st;
            H->ev_in = ml.fork;
            H->ev_out = ml.join;
        }
        if (H->o.profile) {
            H->pev.resize(4 * (size_t)(H->o.nu1 + H->o.nu2), nullptr);
            for (auto &e : H->pev) check_cuda(cudaEventCreate(&e), "cudaEventCreate(profile)");
        }
        {
            SideLane sl = side_get(H->dev);
            H->st2 = sl.st;
            H->ev_fork = sl.fork;
            H->ev_join = sl.join;
        }
        H->sing_host = (int *)pinned_get();
        *H->sing_host = 0;
        enter(*H);
        // levels: N_l = N / 2^l while N_l is even, N_l / 2 >= min_coarse and
        // the coarser level still has interior nodes (Sec. 2.1)
        setup_hierarchy(*H, phi_dev);
        Level &L0 = H->L[0];
        H->u0 = (double *)dalloc(*H, sizeof(double) * split_len(L0.nn), false, false);
        H->npart = (double *)dalloc(*H, sizeof(double) * 4 * (norm_parts(L0) + 1));
        H->ncount = (unsigned *)dalloc(*H, sizeof(unsigned));
        setup_cycle(*H);
        H->nout = (double *)dalloc(*H, sizeof(double) * 4);
        static_assert(sizeof(SolveState) <= kPinBlock && 4 * sizeof(double) <= kPinBlock, "pinned block");
        H->nhost = (double *)pinned_get();
        H->shost = (SolveState *)pinned_get();
        {
            void *alias = nullptr;  // the block's device address (mapped pinned memory)
            if (cudaHostGetDevicePointer(&alias, H->shost, 0) == cudaSuccess) H->shost_dev = (SolveState *)alias;
            else (void)cudaGetLastError();
        }
        H->sdev = (SolveState *)dalloc(*H, sizeof(SolveState));
        set_interior_rhs(*H, L0, f_dev, L0.F);
        for (auto &L : H->L) L.phi = nullptr;
        // the solve graph is captured here, while the device still works on
        // the set-up (capture records launches, it runs nothing)
        if (H->o.use_graph == 1 && !H->o.profile) H->sgraph = build_solve_graph(*H);
        check_cuda(cudaStreamWaitEvent(H->st, H->ev_join, 0), "join wait");  // the coarsest inverse
        check_cuda(cudaStreamSynchronize(H->st), "create sync");
        side_put(H->dev, *H);  // the join is complete: the side lane is idle
        if (*H->sing_host) throw Error{BCMG_EGEOM, "coarsest system is singular"};
        free_temps(*H);
        leave(*H);
    });
    if (rc != BCMG_OK) {
        std::string keep = g_last_error;
        destroy(H);
        g_last_error = keep;
        return rc;
    }
    *out = reinterpret_cast<bcmg_handle>(H);
    return BCMG_OK;
}

int bcmg_destroy(bcmg_handle h) {
    destroy(reinterpret_cast<Handle *>(h));
    return BCMG_OK;
}

int bcmg_ghost_count(bcmg_handle h, int64_t *n) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!n) throw Error{BCMG_EINVAL, "n is null"};
        *n = H.L[0].ng;
    });
}

int bcmg_ghost_points(bcmg_handle h, double *Q) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!Q) throw Error{BCMG_EINVAL, "Q is null"};
        const bool host = is_host_ptr(Q);
        enter(H);
        Level &L = H.L[0];
        if (L.ng > 0)
            check_cuda(cudaMemcpyAsync(Q, L.gQ, sizeof(double) * L.ng * H.d,
                                       host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, H.st),
                       "ghost points copy");
        if (host) check_cuda(cudaStreamSynchronize(H.st), "ghost points sync");  // filled on return
        leave(H);
    });
}

int bcmg_ghost_normals(bcmg_handle h, double *n_dev) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!n_dev) throw Error{BCMG_EINVAL, "n is null"};
        enter(H);
        Level &L = H.L[0];
        // the list holds n axis-major (3 x count); the caller gets count x dim
        for (int a = 0; a < H.d && L.ng > 0; ++a)
            check_cuda(cudaMemcpy2DAsync(n_dev + a, sizeof(double) * H.d, L.gn + (int64_t)a * L.ng, sizeof(double),
                                         sizeof(double), (size_t)L.ng, cudaMemcpyDeviceToDevice, H.st),
                       "ghost normals copy");
        leave(H);
    });
}

int bcmg_set_boundary_values(bcmg_handle h, const double *g) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!g) throw Error{BCMG_EINVAL, "g is null"};
        enter(H);
        Level &L = H.L[0];
        const double *src = g;
        if (is_host_ptr(g) && L.ng > 0) {
            // staged through the level's ghost buffer (idle between calls);
            // the caller's array may be reused on return
            check_cuda(cudaMemcpyAsync(L.gtmp, g, sizeof(double) * L.ng, cudaMemcpyHostToDevice, H.st),
                       "boundary values copy");
            check_cuda(cudaStreamSynchronize(H.st), "boundary values sync");
            src = L.gtmp;
        }
        scatter_ghost_values(H, L, src, L.F);
        leave(H);
    });
}

int bcmg_set_rhs(bcmg_handle h, const double *f_dev) {
    return guarded([&] {
        Handle &H = *checked(h);
        enter(H);
        set_interior_rhs(H, H.L[0], f_dev, H.L[0].F);
        leave(H);
    });
}

int bcmg_vcycle(bcmg_handle h, double *u_dev, int ncycles) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!u_dev || ncycles < 0) throw Error{BCMG_EINVAL, "bad u or ncycles"};
        enter(H);
        copy_active(H, u_dev, H.u0, true);
        for (int c = 0; c < ncycles; ++c) run_vcycle(H);
        copy_active(H, H.u0, u_dev, false);
        leave(H);
    });
}

int bcmg_solve(bcmg_handle h, double *u_dev, double rtol, int max_cycles, int *cycles_done,
               double *final_rel_res) {
    int status = BCMG_OK;
    int rc = guarded([&] {
        Handle &H = *checked(h);
        if (!u_dev || max_cycles < 0 || !(rtol >= 0.0)) throw Error{BCMG_EINVAL, "bad u, rtol or max_cycles"};
        int c = 0;
        double rel = 0.0;
        if (solve_enqueue(H, u_dev, rtol, max_cycles)) status = solve_finish(H, rtol, &c, &rel);
        else status = solve_host_loop(H, u_dev, rtol, max_cycles, &c, &rel);
        if (cycles_done) *cycles_done = c;
        if (final_rel_res) *final_rel_res = rel;
    });
    if (rc != BCMG_OK) return rc;
    return solve_status(status);
}

int bcmg_vcycle_batch(bcmg_handle *handles, double **u_devs, int n, int ncycles) {
    if (n < 0 || (n > 0 && (!handles || !u_devs))) return fail(BCMG_EINVAL, "bad batch arrays");
    return guarded([&] {
        if (ncycles < 0) throw Error{BCMG_EINVAL, "ncycles must be >= 0"};
        std::vector<Handle *> hs = batch_handles(handles, u_devs, n);
        if (batch_eligible(hs)) {
            std::vector<int> cyc(n), st(n);
            std::vector<double> rel(n);
            batched_run(hs, u_devs, 0.0, ncycles, true, cyc.data(), rel.data(), st.data());
            return;
        }
        // each handle's cycles on its own stream, all enqueued before any
        // is waited for
        for (int i = 0; i < n; ++i) {
            Handle &H = *hs[i];
            enter(H);
            copy_active(H, u_devs[i], H.u0, true);
            for (int c = 0; c < ncycles; ++c) run_vcycle(H);
            copy_active(H, H.u0, u_devs[i], false);
            leave(H);
        }
    });
}

int bcmg_solve_batch(bcmg_handle *handles, double **u_devs, int n, double rtol, int max_cycles,
                     int *cycles_done, double *final_rel_res, int *statuses) {
    if (n < 0 || (n > 0 && (!handles || !u_devs))) return fail(BCMG_EINVAL, "bad batch arrays");
    int first = BCMG_OK;
    int rc = guarded([&] {
        if (max_cycles < 0 || !(rtol >= 0.0)) throw Error{BCMG_EINVAL, "bad rtol or max_cycles"};
        std::vector<Handle *> hs = batch_handles(handles, u_devs, n);
        if (batch_eligible(hs)) {
            std::vector<int> cyc(n), st(n);
            std::vector<double> rel(n);
            batched_run(hs, u_devs, rtol, max_cycles, false, cyc.data(), rel.data(), st.data());
            for (int i = 0; i < n; ++i) {
                if (cycles_done) cycles_done[i] = cyc[i];
                if (final_rel_res) final_rel_res[i] = rel[i];
                if (statuses) statuses[i] = st[i];
                if (first == BCMG_OK && st[i] != BCMG_OK) first = st[i];
            }
            return;
        }
        // the solve graphs are built first (no capture while other solves
        // run), then every device-driven solve is enqueued on its handle's
        // own stream before any is waited for, so the solves run concurrently
        for (int i = 0; i < n; ++i) {
            Handle &H = *hs[i];
            if (H.o.use_graph && !H.o.profile && !H.sgraph && !H.sgraph_failed) H.sgraph = build_solve_graph(H);
        }
        std::vector<char> queued(n, 0);
        for (int i = 0; i < n; ++i) queued[i] = solve_enqueue(*hs[i], u_devs[i], rtol, max_cycles) ? 1 : 0;
        for (int i = 0; i < n; ++i) {
            int c = 0;
            double rel = 0.0;
            const int st = queued[i] ? solve_finish(*hs[i], rtol, &c, &rel)
                                     : solve_host_loop(*hs[i], u_devs[i], rtol, max_cycles, &c, &rel);
            if (cycles_done) cycles_done[i] = c;
            if (final_rel_res) final_rel_res[i] = rel;
            if (statuses) statuses[i] = st;
            if (first == BCMG_OK && st != BCMG_OK) first = st;
        }
    });
    if (rc != BCMG_OK) return rc;
    return solve_status(first);
}

int bcmg_dtau_opt(int dim, int bc, int dtau_mode, double dtau_const, double theta, double *out) {
    if (!out) return fail(BCMG_EINVAL, "out is null");
    if ((dim != 2 && dim != 3) || (bc != BCMG_BC_DIRICHLET && bc != BCMG_BC_NEUMANN) || dtau_mode < 0 ||
        dtau_mode > 2 || !(theta >= 0.0 && theta <= 1.0))
        return fail(BCMG_EINVAL, "bad dim, bc, dtau_mode or theta");
    *out = dtau_of(dim, bc, dtau_mode, dtau_const, theta);
    g_last_error.clear();
    return BCMG_OK;
}

int bcmg_workspace_size(bcmg_handle h, int64_t *bytes) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!bytes) throw Error{BCMG_EINVAL, "bytes is null"};
        *bytes = H.alloc_total;
    });
}

int bcmg_debug_live_blocks(int64_t *blocks, int64_t *bytes) {
    if (!blocks || !bytes) return fail(BCMG_EINVAL, "null pointer");
    *blocks = g_live_blocks.load();
    *bytes = g_live_bytes.load();
    g_last_error.clear();
    return BCMG_OK;
}

int bcmg_batch_last_shape(int *block, int *items, int64_t *tail_rows) {
    if (!block || !items || !tail_rows) return fail(BCMG_EINVAL, "null pointer");
    bcmg::batch_last_shape(block, items, tail_rows);
    g_last_error.clear();
    return BCMG_OK;
}

int bcmg_debug_batch_shape(int block, int items, int64_t tail_rows) {
    if (block != 0 && block != 64 && block != 128 && block != 256)
        return fail(BCMG_EINVAL, "block must be 0, 64, 128 or 256");
    if (items != 1 && items != 4) return fail(BCMG_EINVAL, "items must be 1 or 4");
    if (tail_rows < 0) return fail(BCMG_EINVAL, "tail_rows must be >= 0");
    bcmg::batch_shape_override(block, items, tail_rows);
    g_last_error.clear();
    return BCMG_OK;
}

int bcmg_debug_fail_allocation(int64_t k) {
    if (k < 0) return fail(BCMG_EINVAL, "k must be >= 0");
    g_fail_countdown.store(k);
    g_last_error.clear();
    return BCMG_OK;
}

int bcmg_memory_footprint(bcmg_handle h, int64_t *bytes) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!bytes) throw Error{BCMG_EINVAL, "bytes is null"};
        *bytes = H.dev_bytes;
    });
}

int bcmg_footprint(int dim, const int64_t *N, const bcmg_opts *opts, size_t *bytes) {
    if (!N || !bytes) return fail(BCMG_EINVAL, "null pointer");
    if (dim != 2 && dim != 3) return fail(BCMG_EINVAL, "bad dim");
    for (int a = 1; a < dim; ++a)
        if (N[a] != N[0]) return fail(BCMG_EINVAL, "grids are cubic: every N[a] must equal N[0]");
    int64_t b = 0;
    const int rc = bcmg_footprint_estimate(dim, N[0], opts, &b);
    if (rc == BCMG_OK) *bytes = (size_t)b;
    return rc;
}

int bcmg_footprint_estimate(int dim, int64_t N, const bcmg_opts *opts, int64_t *bytes) {
    if (!bytes) return fail(BCMG_EINVAL, "bytes is null");
    if ((dim != 2 && dim != 3) || N < 4 || N > 65534) return fail(BCMG_EINVAL, "bad dim or N");
    bcmg_opts o;
    if (opts) o = *opts;
    else bcmg_default_opts(&o);
    // dense per-level arrays (class byte, u, F, its scaled copy, r; FP32
    // u, F, scaled F, r for the mixed path) over the levels the coarsening
    // rule allows, doubled to cover the compacted lists (ghost weights,
    // expanded extension), which hold far fewer entries than the grid but
    // more bytes per entry
    const double per_node = 1.0 + 4.0 * 8.0 + (o.precision == BCMG_PREC_MIXED ? 4.0 * 4.0 : 0.0);
    double total = 0.0;
    int64_t Nl = N;
    for (int l = 0; l < std::max(o.max_levels, 1); ++l) {
        total += std::pow((double)(Nl + 1), dim) * per_node;
        if (Nl % 2 != 0 || Nl / 2 < o.min_coarse) break;
        Nl /= 2;
    }
    // plus the chunks small arrays are carved from (a few per hierarchy)
    *bytes = (int64_t)(2.0 * total) + 3 * (int64_t)(4 << 20);
    g_last_error.clear();
    return BCMG_OK;
}

int bcmg_residual_norm(bcmg_handle h, const double *u_dev, double *out_host) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!u_dev || !out_host) throw Error{BCMG_EINVAL, "null pointer"};
        enter(H);
        copy_active(H, u_dev, H.u0, true);
        enqueue_norms(H);
        fetch_norms(H, out_host);
        leave(H);
    });
}

const char *bcmg_last_error(void) { return g_last_error.c_str(); }

int64_t bcmg_kernel_launches(void) { return launches_total(); }

int bcmg_profile_read(bcmg_handle h, double *out_host) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!out_host) throw Error{BCMG_EINVAL, "null pointer"};
        out_host[0] = H.prof_ms;
        out_host[1] = (double)H.prof_n;
    });
}

int bcmg_time_sweeps(bcmg_handle h, int nsweeps, double *ms_host) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!ms_host || nsweeps < 1) throw Error{BCMG_EINVAL, "bad argument"};
        if (H.o.ordering != BCMG_ORDER_RB) throw Error{BCMG_EINVAL, "red-black ordering only"};
        enter(H);
        *ms_host = time_sweeps(H, nsweeps);
        leave(H);
    });
}

int bcmg_time_sweeps_bf16(bcmg_handle h, int nsweeps, double *ms_host) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!ms_host || nsweeps < 1) throw Error{BCMG_EINVAL, "bad argument"};
        if (H.o.ordering != BCMG_ORDER_RB) throw Error{BCMG_EINVAL, "red-black ordering only"};
        enter(H);
        *ms_host = time_sweeps_bf16(H, nsweeps);
        leave(H);
    });
}

int bcmg_num_levels(bcmg_handle h, int *levels) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!levels) throw Error{BCMG_EINVAL, "null pointer"};
        *levels = (int)H.L.size();
    });
}

int bcmg_level_info(bcmg_handle h, int level, int64_t *out) {
    return guarded([&] {
        Handle &H = *checked(h);
        Level &L = level_of(H, level);
        if (!out) throw Error{BCMG_EINVAL, "null pointer"};
        int64_t v[10] = {L.N, L.n, L.nn, L.nint, L.ng, L.nb, L.nbox, L.nclamp, L.nfall, L.nact};
        std::memcpy(out, v, sizeof(v));
    });
}

int bcmg_level_lists(bcmg_handle h, int level, int64_t *out) {
    return guarded([&] {
        Handle &H = *checked(h);
        Level &L = level_of(H, level);
        if (!out) throw Error{BCMG_EINVAL, "null pointer"};
        const int64_t v[3] = {L.nred, L.nbn, L.nint - L.nred - L.nbn};
        std::memcpy(out, v, sizeof(v));
    });
}

int bcmg_get_class(bcmg_handle h, int level, uint8_t *cls_host) {
    return guarded([&] {
        Handle &H = *checked(h);
        Level &L = level_of(H, level);
        if (!cls_host) throw Error{BCMG_EINVAL, "null pointer"};
        check_cuda(cudaMemcpyAsync(cls_host, L.cls, L.nn, cudaMemcpyDeviceToHost, H.st), "class copy");
        check_cuda(cudaStreamSynchronize(H.st), "class sync");
    });
}

int bcmg_get_ghosts(bcmg_handle h, int level, int64_t *idx, double *eta, double *n3, double *xi3, int32_t *s3,
                    int32_t *q3, double *dtau, double *Q3) {
    return guarded([&] {
        Handle &H = *checked(h);
        Level &L = level_of(H, level);
        const int64_t ng = L.ng;
        const int d = H.d;
        std::vector<uint32_t> gi(ng);
        std::vector<uint16_t> gc(ng);
        std::vector<double> xi(3 * ng), nn(3 * ng), et(ng), dt(ng), Q(d * ng);
        if (ng > 0) {
            check_cuda(cudaMemcpyAsync(gi.data(), L.gidx, 4 * ng, cudaMemcpyDeviceToHost, H.st), "g");
            check_cuda(cudaMemcpyAsync(gc.data(), L.gcode, 2 * ng, cudaMemcpyDeviceToHost, H.st), "g");
            check_cuda(cudaMemcpyAsync(xi.data(), L.gxi, 8 * 3 * ng, cudaMemcpyDeviceToHost, H.st), "g");
            check_cuda(cudaMemcpyAsync(nn.data(), L.gn, 8 * 3 * ng, cudaMemcpyDeviceToHost, H.st), "g");
            check_cuda(cudaMemcpyAsync(et.data(), L.geta, 8 * ng, cudaMemcpyDeviceToHost, H.st), "g");
            check_cuda(cudaMemcpyAsync(dt.data(), L.gdt, 8 * ng, cudaMemcpyDeviceToHost, H.st), "g");
            check_cuda(cudaMemcpyAsync(Q.data(), L.gQ, 8 * d * ng, cudaMemcpyDeviceToHost, H.st), "g");
        }
        check_cuda(cudaStreamSynchronize(H.st), "ghost sync");
        for (int64_t g = 0; g < ng; ++g) {
            if (idx) idx[g] = gi[g];
            if (eta) eta[g] = et[g];
            if (dtau) dtau[g] = dt[g];
            for (int a = 0; a < 3; ++a) {
                const bool on = a < d;
                if (n3) n3[3 * g + a] = on ? nn[a * ng + g] : 0.0;
                if (xi3) xi3[3 * g + a] = on ? xi[a * ng + g] : 0.0;
                if (s3) s3[3 * g + a] = on ? (((gc[g] >> a) & 1) ? -1 : 1) : 0;
                if (q3) q3[3 * g + a] = on ? ((gc[g] >> (3 + 2 * a)) & 3) : 0;
                if (Q3) Q3[3 * g + a] = on ? Q[g * d + a] : 0.0;
            }
        }
    });
}

int bcmg_get_band(bcmg_handle h, int level, int64_t *idx_host) {
    return guarded([&] {
        Handle &H = *checked(h);
        Level &L = level_of(H, level);
        if (!idx_host) throw Error{BCMG_EINVAL, "null pointer"};
        std::vector<uint32_t> b(L.nb);
        if (L.nb > 0)
            check_cuda(cudaMemcpyAsync(b.data(), L.bidx, 4 * L.nb, cudaMemcpyDeviceToHost, H.st), "band copy");
        check_cuda(cudaStreamSynchronize(H.st), "band sync");
        for (int64_t i = 0; i < L.nb; ++i) idx_host[i] = b[i];
    });
}

int bcmg_smooth(bcmg_handle h, int level, double *u_dev, const double *F_dev, int nsteps) {
    return guarded([&] {
        Handle &H = *checked(h);
        Level &L = level_of(H, level);
        if (!u_dev || !F_dev || nsteps < 0) throw Error{BCMG_EINVAL, "bad argument"};
        enter(H);
        double *u = stage_buf(H, 0), *F = stage_buf(H, 1);
        dense_to_split(H, L, u_dev, u);
        dense_to_split(H, L, F_dev, F);
        smooth(H, L, u, (const double *)F, nsteps);
        split_to_dense(H, L, u, u_dev);
        leave(H);
    });
}

int bcmg_residual(bcmg_handle h, int level, const double *u_dev, const double *F_dev, double *r_dev) {
    return guarded([&] {
        Handle &H = *checked(h);
        Level &L = level_of(H, level);
        if (!u_dev || !F_dev || !r_dev) throw Error{BCMG_EINVAL, "bad argument"};
        enter(H);
        double *u = stage_buf(H, 0), *F = stage_buf(H, 1), *r = stage_buf(H, 2);
        dense_to_split(H, L, u_dev, u);
        dense_to_split(H, L, F_dev, F);
        dense_to_split(H, L, r_dev, r);
        residual(H, L, (const double *)u, (const double *)F, r);
        split_to_dense(H, L, r, r_dev);
        leave(H);
    });
}

int bcmg_extend(bcmg_handle h, int level, double *a_dev) {
    return guarded([&] {
        Handle &H = *checked(h);
        Level &L = level_of(H, level);
        if (!a_dev) throw Error{BCMG_EINVAL, "bad argument"};
        enter(H);
        double *a = stage_buf(H, 0);
        dense_to_split(H, L, a_dev, a);
        extend(H, L, a);
        split_to_dense(H, L, a, a_dev);
        leave(H);
    });
}

int bcmg_restrict(bcmg_handle h, int level, const double *r_fine_dev, double *F_coarse_dev) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (level < 0 || level + 1 >= (int)H.L.size()) throw Error{BCMG_EINVAL, "level out of range"};
        if (!r_fine_dev || !F_coarse_dev) throw Error{BCMG_EINVAL, "bad argument"};
        enter(H);
        Level &Lf = H.L[level], &Lc = H.L[level + 1];
        double *rf = stage_buf(H, 0), *Fc = stage_buf(H, 1);
        dense_to_split(H, Lf, r_fine_dev, rf);
        dense_to_split(H, Lc, F_coarse_dev, Fc);
        restrict_to<double>(H, Lf, Lc, (const double *)rf, Fc, nullptr);
        split_to_dense(H, Lc, Fc, F_coarse_dev);
        leave(H);
    });
}

int bcmg_prolong(bcmg_handle h, int level, const double *e_coarse_dev, double *u_fine_dev) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (level < 0 || level + 1 >= (int)H.L.size()) throw Error{BCMG_EINVAL, "level out of range"};
        if (!e_coarse_dev || !u_fine_dev) throw Error{BCMG_EINVAL, "bad argument"};
        enter(H);
        Level &Lf = H.L[level], &Lc = H.L[level + 1];
        double *ec = stage_buf(H, 0), *uf = stage_buf(H, 1);
        dense_to_split(H, Lc, e_coarse_dev, ec);
        dense_to_split(H, Lf, u_fine_dev, uf);
        prolong(H, Lf, Lc, (const double *)ec, uf);
        split_to_dense(H, Lf, uf, u_fine_dev);
        leave(H);
    });
}

int bcmg_coarsest_solve(bcmg_handle h, double *u_dev, const double *F_dev) {
    return guarded([&] {
        Handle &H = *checked(h);
        if (!u_dev || !F_dev) throw Error{BCMG_EINVAL, "bad argument"};
        enter(H);
        Level &L = H.L.back();
        double *u = stage_buf(H, 0), *F = stage_buf(H, 1);
        dense_to_split(H, L, u_dev, u);
        dense_to_split(H, L, F_dev, F);
        coarsest_correct(H, L, u, (const double *)F);
        split_to_dense(H, L, u, u_dev);
        leave(H);
    });
}

}  // extern "C"
