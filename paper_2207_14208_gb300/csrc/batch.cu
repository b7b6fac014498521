// Batched solves: many hierarchies of different sizes and shapes advance
// together, one launch per stage of the V-cycle for all of them.
//
// A batch is a set of hierarchies of one dimension and working precision
// (red-black V-cycles, expanded extensions).  Their levels are listed in a
// device table (one descriptor per hierarchy and level, the levels of a
// hierarchy consecutive) and every stage of the cycle -- a colour sweep, the
// ghost relaxation, the residual, the extension, the restriction, the
// prolongation, the coarsest solve -- is one launch whose blocks a task map
// assigns to (level descriptor, block within that level's list).  Levels are
// aligned by depth: at depth k the hierarchies with a level k above their
// coarsest smooth and restrict, those whose coarsest level is k solve it.
// The coarse levels that a single hierarchy runs in its thread-block-cluster
// tail run here as ordinary stages, shared by the batch.  Each hierarchy
// keeps its own convergence state on the device; once it has converged (or
// hit its limit) its blocks return before the dependency wait, and the
// whole solve -- initial norms, then a WHILE loop of (cycle, norms, check)
// -- is one CUDA graph whose condition is "some hierarchy still runs".  The
// launch shape of the stages is chosen by measurement (a small autotuner):
// one batched cycle is timed for block sizes of 64, 128 and 256 threads,
// each with one or four items per thread in the node-parallel stages, and
// the fastest kept for batches of the same shape.  Several items per thread
// put several independent load chains of a thread in flight at once: a
// block's work is a short chain of dependent loads (task map, list entry,
// neighbours), so on the large levels one item per thread leaves the memory
// system idle between waves of blocks.
//
// Every node is updated by the same device functions as in a single solve
// (nodeops.cuh).  The differences from a single solve are the coarse levels,
// which the cluster tail sums in a different order (the tail's ghost rows are
// split over four lanes), so results agree with single solves to rounding
// (and with the oracle to its tolerance), not bit for bit.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "bcmg_internal.cuh"
#include "nodeops.cuh"

namespace bcmg {
namespace {

template <typename T>
struct BLev {
    G2 g;
    const uint32_t *ilist;
    int64_t nred, nint;
    const uint32_t *gidx;
    const uint16_t *gcode;
    const T *gw;
    const double *gdt;
    int64_t ng;
    const uint32_t *bidx;
    const uint8_t *ecnt;
    const uint32_t *eg;
    const double *ew;
    int64_t nb;
    const uint32_t *fmask;
    T *u, *F, *Fs, *r, *tmp;
    const uint32_t *act;
    int64_t nact;
    const double *Ainv;
    double *crhs;
    int h;  // hierarchy
};

struct BTask {
    uint32_t lev;  // level descriptor
    uint32_t blk;  // block within the level's list
    uint32_t sub;  // residual: 0 interior rows, 1 ghost rows
    uint32_t pad;
};

// A stage's blocks by level: range k covers blocks [begin_k, begin_{k+1})
// of level descriptor lev (the part sub of its rows)
struct BRange {
    uint32_t lev, sub, begin, pad;
};

// the task of this block: the last range that begins at or before it
// (binary search over the stage's few ranges; fixed tables, read before the
// dependency wait)
__device__ __forceinline__ BTask block_task(const BRange *__restrict__ rg, int nr) {
    const uint32_t b = blockIdx.x;
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rg[mid].begin <= b) lo = mid;
        else hi = mid - 1;
    }
    const BRange r = rg[lo];
    return BTask{r.lev, b - r.begin, r.sub, 0u};
}

// per-hierarchy state of a batched solve (device)
struct BCtl {
    double rtol;
    int max_cycles;
    int cycles;
    double r0, rel;
    int status;
    int done;
    int fixed;  // run exactly max_cycles (batched V-cycles), whatever the residual
};

struct BShared {  // batch-wide counters of the check kernel
    unsigned blocks_done;
    unsigned active;
};

__device__ __forceinline__ bool bdone(const BCtl *ctl, int h) { return *(volatile const int *)&ctl[h].done; }

// Entry of a stage kernel after its fixed-table prologue; true when the
// block is to return because its hierarchy has finished.  The flag was
// written by the check that ends a cycle, in an earlier launch of the loop
// body (or before the graph), which completed before this launch began, so
// it is read before the dependency wait (a volatile load, served by L2) and
// a finished hierarchy's block leaves without waiting.  Block 0 always
// waits: every grid then completes only after its predecessor, and starts
// only after its predecessor's block 0 has passed the wait, so the ordering
// pdl_begin relies on holds even for a stage whose hierarchies have all
// finished.
__device__ __forceinline__ bool bskip(const BCtl *ctl, int h) {
    const bool d = bdone(ctl, h);
    if (d && blockIdx.x != 0) return true;
    pdl_begin();
    return d;
}

// item j of this thread when a block takes NPT items per thread (strided by
// the block size, so a warp's loads of one item index stay contiguous)
template <int NPT>
__device__ __forceinline__ int64_t bitem(const BTask &t, int j) {
    return ((int64_t)t.blk * NPT + j) * blockDim.x + threadIdx.x;
}

// One colour sweep, NPT nodes per thread: every load of the thread's nodes
// is issued before its first store (a colour sweep reads only the other
// colour, so the nodes of a thread never depend on one another).
template <int D, typename T, int NPT>
__global__ void __launch_bounds__(kT) kb_smooth(const BLev<T> *__restrict__ lv, const BRange *__restrict__ rg, int nr,
                                                const BCtl *__restrict__ ctl, int colour) {
    const BTask t = block_task(rg, nr);
    const BLev<T> &A = lv[t.lev];
    const G2 G = A.g;
    const int64_t n = colour ? A.nint - A.nred : A.nred;
    const uint32_t *list = A.ilist + (colour ? A.nred : 0);
    uint32_t X[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t i = bitem<NPT>(t, j);
        X[j] = i < n ? list[i] : 0u;
    }
    T *u = A.u;
    const T *Fs = A.Fs;
    if (bskip(ctl, A.h)) return;
    const bool par = (G.n & 1) && G.lay.s == 1;
    T s[NPT], f[NPT];
    int64_t x[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        s[j] = f[j] = T(0);
        x[j] = 0;
        if (bitem<NPT>(t, j) >= n) continue;
        if (par) {
            s[j] = nbr_sum_par<D, T>(X[j], u, G, colour, x[j]);
        } else {
            s[j] = nbr_sum<D, T>(u, X[j], G);
            x[j] = pos(X[j], G.lay);
        }
        f[j] = Fs[x[j]];
    }
#pragma unroll
    for (int j = 0; j < NPT; ++j)
        if (bitem<NPT>(t, j) < n) u[x[j]] = fma(s[j], (T)G.inv_diag, f[j]);
}

template <int D, typename T>
__global__ void __launch_bounds__(kT) kb_ghost_relax(const BLev<T> *__restrict__ lv, const BRange *__restrict__ rg, int nr,
                                                     const BCtl *__restrict__ ctl) {
    const BTask t = block_task(rg, nr);
    const BLev<T> &A = lv[t.lev];
    const G2 G = A.g;
    const int64_t ng = A.ng;
    const int64_t g = (int64_t)t.blk * blockDim.x + threadIdx.x;
    const bool on = g < ng;
    const int64_t X = on ? A.gidx[g] : 0;
    const uint16_t code = on ? A.gcode[g] : 0;
    const T dt = on ? (T)A.gdt[g] : T(0);
    T w[(D == 3) ? 27 : 9];
    ghost_weights<D, T>(code, A.gw, ng, on ? g : 0, w);
    const T *u = A.u, *F = A.F;
    T *tmp = A.tmp;
    if (bskip(ctl, A.h) || !on) return;
    const int64_t x = pos(X, G.lay);
    tmp[g] = fma(dt, F[x] - ghost_Bw<D, T>(X, code, w, u, G), u[x]);
}

template <typename T>
__global__ void __launch_bounds__(kT) kb_ghost_scatter(const BLev<T> *__restrict__ lv, const BRange *__restrict__ rg, int nr,
                                                       const BCtl *__restrict__ ctl) {
    const BTask t = block_task(rg, nr);
    const BLev<T> &A = lv[t.lev];
    const int64_t g = (int64_t)t.blk * blockDim.x + threadIdx.x;
    const bool on = g < A.ng;
    const uint32_t X = on ? A.gidx[g] : 0u;
    const Lay ly = A.g.lay;
    const T *tmp = A.tmp;
    T *u = A.u;
    if (bskip(ctl, A.h) || !on) return;
    u[pos(X, ly)] = tmp[g];
}

// residual rows: interior rows (sub 0, NPT rows per thread) or ghost rows
// (sub 1, one row per thread); with part, every block writes its norm
// partials at its launch slot (a finished hierarchy's slots are left as they
// are: the check does not read them)
template <int D, typename T, int NPT>
__global__ void __launch_bounds__(kT) kb_residual(const BLev<T> *__restrict__ lv, const BRange *__restrict__ rg, int nr,
                                                  const BCtl *__restrict__ ctl, double *__restrict__ part) {
    const BTask t = block_task(rg, nr);
    const BLev<T> &A = lv[t.lev];
    const G2 G = A.g;
    const T *u = A.u, *F = A.F;
    T *r = A.r;
    double s2 = 0.0;
    long long mxb = 0;
    if (t.sub != 0) {  // ghost rows
        const int64_t i = (int64_t)t.blk * blockDim.x + threadIdx.x;
        const bool on = i < A.ng;
        const int64_t X = on ? A.gidx[i] : 0;
        const uint16_t code = on ? A.gcode[i] : 0;
        T w[(D == 3) ? 27 : 9];
        ghost_weights<D, T>(code, A.gw, A.ng, on ? i : 0, w);
        if (bskip(ctl, A.h)) return;  // uniform over the block (one hierarchy)
        if (on) {
            const int64_t x = pos(X, G.lay);
            const T v = F[x] - ghost_Bw<D, T>(X, code, w, u, G);
            r[x] = v;
            s2 = (double)v * (double)v;
            mxb = abs_bits((double)v);
        }
        if (part) block_partials(s2, mxb, part, blockIdx.x, false);
        return;
    }
    const int64_t nint = A.nint;
    uint32_t X[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t i = bitem<NPT>(t, j);
        X[j] = i < nint ? A.ilist[i] : 0u;
    }
    if (bskip(ctl, A.h)) return;
    T v[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) v[j] = bitem<NPT>(t, j) < nint ? residual_int<D, T>(X[j], u, F, G) : T(0);
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        if (bitem<NPT>(t, j) >= nint) continue;
        r[pos(X[j], G.lay)] = v[j];
        s2 = fma((double)v[j], (double)v[j], s2);
        mxb = max(mxb, abs_bits((double)v[j]));
    }
    if (part) block_partials(s2, mxb, part, blockIdx.x, true);
}

// expanded extension of the level's r (which = 0) or u (which = 1) into its band
template <typename T>
__global__ void __launch_bounds__(kT) kb_extend(const BLev<T> *__restrict__ lv, const BRange *__restrict__ rg, int nr,
                                                const BCtl *__restrict__ ctl, int which) {
    const BTask t = block_task(rg, nr);
    const BLev<T> &A = lv[t.lev];
    const int64_t nb = A.nb;
    const int64_t b = (int64_t)t.blk * blockDim.x + threadIdx.x;
    const bool on = b < nb;
    const uint32_t X = on ? A.bidx[b] : 0u;
    const uint32_t *eg = A.eg;
    const double *ew = A.ew;
    EllRound<T> R;
    R.c = 0;
    if (on) ell_first<T>(b, A.ecnt, eg, ew, nb, R);
    T *a = which ? A.u : A.r;
    const Lay ly = A.g.lay;
    if (bskip(ctl, A.h) || !on) return;
    a[pos(X, ly)] = extend_from<T>(b, R, eg, ew, nb, a, ly);
}

// restriction to the coarse level t.lev from the fine level t.lev - 1 (rows:
// coarse interior rows, then coarse ghost rows; NPT rows per thread); the
// coarse correction is zeroed on the same rows
template <int D, typename T, int NPT>
__global__ void __launch_bounds__(kT) kb_restrict(const BLev<T> *__restrict__ lv, const BRange *__restrict__ rg, int nr,
                                                  const BCtl *__restrict__ ctl) {
    const BTask t = block_task(rg, nr);
    const BLev<T> &C = lv[t.lev];
    const BLev<T> &Fl = lv[t.lev - 1];
    const G2 Gc = C.g, Gf = Fl.g;
    const int64_t nint_c = C.nint, nrow = C.nint + C.ng;
    uint32_t Xc[NPT], mask[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t row = bitem<NPT>(t, j);
        const bool on = row < nrow;
        Xc[j] = on ? (row < nint_c ? C.ilist[row] : C.gidx[row - nint_c]) : 0u;
        mask[j] = on ? C.fmask[row] : 0u;
    }
    const T *rf = Fl.r;
    T *Fc = C.F, *Fsc = C.Fs, *uc = C.u;
    if (bskip(ctl, C.h)) return;
    T fc[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        int ic[3];
        coords(Xc[j], (uint32_t)Gc.n, D, ic);
        fc[j] = bitem<NPT>(t, j) < nrow ? restrict_masked<D, T>(ic, mask[j], rf, Gf) : T(0);
    }
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t row = bitem<NPT>(t, j);
        if (row >= nrow) continue;
        const int64_t xc = pos(Xc[j], Gc.lay);
        Fc[xc] = fc[j];
        if (row < nint_c) Fsc[xc] = scaled_rhs<T>(fc[j], Gc);
        uc[xc] = T(0);
    }
}

// prolongation into the fine level t.lev from t.lev + 1 (rows: interior
// rows, then ghost rows; NPT rows per thread)
template <int D, typename T, int NPT>
__global__ void __launch_bounds__(kT) kb_prolong(const BLev<T> *__restrict__ lv, const BRange *__restrict__ rg, int nr,
                                                 const BCtl *__restrict__ ctl) {
    const BTask t = block_task(rg, nr);
    const BLev<T> &Fl = lv[t.lev];
    const BLev<T> &C = lv[t.lev + 1];
    const G2 Gf = Fl.g, Gc = C.g;
    const int64_t nint = Fl.nint, nrow = Fl.nint + Fl.ng;
    uint32_t X[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t i = bitem<NPT>(t, j);
        X[j] = i < nrow ? (i < nint ? Fl.ilist[i] : Fl.gidx[i - nint]) : 0u;
    }
    const T *ec = C.u;
    T *uf = Fl.u;
    if (bskip(ctl, Fl.h)) return;
    T v[NPT];
    int64_t x[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        v[j] = T(0);
        x[j] = pos(X[j], Gf.lay);
        if (bitem<NPT>(t, j) >= nrow) continue;
        int iy[3];
        coords(X[j], (uint32_t)Gf.n, D, iy);
        v[j] = uf[x[j]] + prolong_at<D, T>(iy, ec, Gc);
    }
#pragma unroll
    for (int j = 0; j < NPT; ++j)
        if (bitem<NPT>(t, j) < nrow) uf[x[j]] = v[j];
}

template <typename T>
__global__ void __launch_bounds__(kT) kb_coarse_gather(const BLev<T> *__restrict__ lv, const BRange *__restrict__ rg, int nr,
                                                       const BCtl *__restrict__ ctl) {
    const BTask t = block_task(rg, nr);
    const BLev<T> &A = lv[t.lev];
    const int64_t j = (int64_t)t.blk * blockDim.x + threadIdx.x;
    const bool on = j < A.nact;
    const uint32_t X = on ? A.act[j] : 0u;
    const Lay ly = A.g.lay;
    const T *r = A.r;
    double *rhs = A.crhs;
    if (bskip(ctl, A.h) || !on) return;
    rhs[j] = (double)r[pos(X, ly)];
}

// u[act[i]] += (A^-1 rhs)_i, one warp per row (FP64 accumulation)
template <typename T>
__global__ void __launch_bounds__(kT) kb_coarse_gemv(const BLev<T> *__restrict__ lv, const BRange *__restrict__ rg, int nr,
                                                     const BCtl *__restrict__ ctl) {
    const BTask t = block_task(rg, nr);
    const BLev<T> &A = lv[t.lev];
    const int64_t nact = A.nact;
    const double *Ainv = A.Ainv, *rhs = A.crhs;
    const Lay ly = A.g.lay;
    T *u = A.u;
    const uint32_t *act = A.act;
    if (bskip(ctl, A.h)) return;
    const int64_t i = (int64_t)t.blk * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (i >= nact) return;
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int64_t j = lane; j < nact; j += 32) s = fma(Ainv[i * nact + j], rhs[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) u[pos(act[i], ly)] += (T)s;
}

// start of a refinement step on the finest level: F32 = (float) r64, the
// scaled copy on interior rows, e32 = 0 (level entries of the FP64 and FP32
// tables are the same index); NPT rows per thread
template <int NPT>
__global__ void __launch_bounds__(kT) kb_ir_begin(const BLev<double> *__restrict__ l64,
                                                  const BLev<float> *__restrict__ l32,
                                                  const BRange *__restrict__ rg, int nr, const BCtl *__restrict__ ctl) {
    const BTask t = block_task(rg, nr);
    const BLev<double> &A = l64[t.lev];
    const BLev<float> &B = l32[t.lev];
    const G2 G = A.g;
    const int64_t nint = A.nint, nrow = A.nint + A.ng;
    uint32_t X[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t i = bitem<NPT>(t, j);
        X[j] = i < nrow ? (i < nint ? A.ilist[i] : A.gidx[i - nint]) : 0u;
    }
    const double *r = A.r;
    float *F32 = B.F, *Fs32 = B.Fs, *e32 = B.u;
    if (bskip(ctl, A.h)) return;
    float f[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) f[j] = bitem<NPT>(t, j) < nrow ? (float)r[pos(X[j], G.lay)] : 0.0f;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t i = bitem<NPT>(t, j);
        if (i >= nrow) continue;
        const int64_t x = pos(X[j], G.lay);
        F32[x] = f[j];
        if (i < nint) Fs32[x] = scaled_rhs<float>(f[j], G);
        e32[x] = 0.0f;
    }
}

// end of a refinement step: u += e on interior and ghost rows (FP64)
template <int NPT>
__global__ void __launch_bounds__(kT) kb_ir_update(const BLev<double> *__restrict__ l64,
                                                   const BLev<float> *__restrict__ l32,
                                                   const BRange *__restrict__ rg, int nr, const BCtl *__restrict__ ctl) {
    const BTask t = block_task(rg, nr);
    const BLev<double> &A = l64[t.lev];
    const BLev<float> &B = l32[t.lev];
    const int64_t nint = A.nint, nrow = A.nint + A.ng;
    uint32_t X[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t i = bitem<NPT>(t, j);
        X[j] = i < nrow ? (i < nint ? A.ilist[i] : A.gidx[i - nint]) : 0u;
    }
    const Lay ly = A.g.lay;
    const float *e32 = B.u;
    double *u = A.u;
    if (bskip(ctl, A.h)) return;
    double v[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t x = pos(X[j], ly);
        v[j] = bitem<NPT>(t, j) < nrow ? u[x] + (double)e32[x] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < NPT; ++j)
        if (bitem<NPT>(t, j) < nrow) u[pos(X[j], ly)] = v[j];
}

// ------------------------------------------------------------ block tail
// The coarse levels of a hierarchy in one block: the levels from the tail's
// top down to the coarsest, every stage of the cycle on them as a phase of
// the block, phases separated by the block barrier.  Per node the same
// device functions as the stage kernels, in the same phase order, so the
// results are those of the stage path.  One launch (one block per
// hierarchy with a tail) replaces the seventeen or so stage launches per
// coarse level.  Lists of a tail level are walked in chunks of kBTEnt
// entries per thread, every load of a chunk before its first store.
constexpr int kBT = 256;     // threads of a tail block (two blocks per SM)
constexpr int kBTEnt = 4;    // entries per thread and chunk
constexpr int64_t kBTMaxCoarse = 192;  // coarsest unknowns of a tail (its dense GEMV runs on one SM)

struct BTail {
    uint32_t lev0;  // level descriptor of the tail's top level
    uint32_t nl;    // tail levels (the last one is the coarsest)
};

__device__ __forceinline__ int64_t bt_entry(int64_t b0, int j) {
    return b0 + (int64_t)j * blockDim.x + threadIdx.x;
}

template <int D, typename T>
__device__ void bt_sweep(const BLev<T> &A, int colour) {
    const G2 G = A.g;
    const int64_t n = colour ? A.nint - A.nred : A.nred;
    const uint32_t *list = A.ilist + (colour ? A.nred : 0);
    T *const u = A.u;
    const T *const Fs = A.Fs;
    const bool par = (G.n & 1) && G.lay.s == 1;
    for (int64_t b0 = 0; b0 < n; b0 += (int64_t)kBTEnt * blockDim.x) {
        uint32_t X[kBTEnt];
#pragma unroll
        for (int j = 0; j < kBTEnt; ++j) X[j] = bt_entry(b0, j) < n ? list[bt_entry(b0, j)] : 0u;
        T s[kBTEnt], f[kBTEnt];
        int64_t x[kBTEnt];
#pragma unroll
        for (int j = 0; j < kBTEnt; ++j) {
            s[j] = f[j] = T(0);
            x[j] = 0;
            if (bt_entry(b0, j) >= n) continue;
            if (par) {
                s[j] = nbr_sum_par<D, T>(X[j], u, G, colour, x[j]);
            } else {
                s[j] = nbr_sum<D, T>(u, X[j], G);
                x[j] = pos(X[j], G.lay);
            }
            f[j] = Fs[x[j]];
        }
#pragma unroll
        for (int j = 0; j < kBTEnt; ++j)
            if (bt_entry(b0, j) < n) u[x[j]] = fma(s[j], (T)G.inv_diag, f[j]);
    }
    __syncthreads();
}

// ghost relaxation from the same u, then the write-back
template <int D, typename T>
__device__ void bt_relax(const BLev<T> &A) {
    const G2 G = A.g;
    const int64_t ng = A.ng;
    const T *const F = A.F;
    T *const u = A.u;
    T *const tmp = A.tmp;
    const uint32_t *const gidx = A.gidx;
    const uint16_t *const gcode = A.gcode;
    const double *const gdt = A.gdt;
    const T *const gw = A.gw;
    for (int64_t g = threadIdx.x; g < ng; g += blockDim.x) {
        const int64_t X = gidx[g];
        const uint16_t code = gcode[g];
        const T dt = (T)gdt[g];
        T w[(D == 3) ? 27 : 9];
        ghost_weights<D, T>(code, gw, ng, g, w);
        const int64_t x = pos(X, G.lay);
        tmp[g] = fma(dt, F[x] - ghost_Bw<D, T>(X, code, w, u, G), u[x]);
    }
    __syncthreads();
    for (int64_t g = threadIdx.x; g < ng; g += blockDim.x) u[pos(gidx[g], G.lay)] = tmp[g];
    __syncthreads();
}

template <int D, typename T>
__device__ void bt_residual(const BLev<T> &A) {
    const G2 G = A.g;
    const int64_t nint = A.nint, ng = A.ng;
    const T *const u = A.u, *const F = A.F;
    T *const r = A.r;
    const uint32_t *const ilist = A.ilist, *const gidx = A.gidx;
    const uint16_t *const gcode = A.gcode;
    const T *const gw = A.gw;
    for (int64_t b0 = 0; b0 < nint; b0 += (int64_t)kBTEnt * blockDim.x) {
        uint32_t X[kBTEnt];
#pragma unroll
        for (int j = 0; j < kBTEnt; ++j) X[j] = bt_entry(b0, j) < nint ? ilist[bt_entry(b0, j)] : 0u;
        T v[kBTEnt];
#pragma unroll
        for (int j = 0; j < kBTEnt; ++j) v[j] = bt_entry(b0, j) < nint ? residual_int<D, T>(X[j], u, F, G) : T(0);
#pragma unroll
        for (int j = 0; j < kBTEnt; ++j)
            if (bt_entry(b0, j) < nint) r[pos(X[j], G.lay)] = v[j];
    }
    for (int64_t g = threadIdx.x; g < ng; g += blockDim.x) {
        const int64_t X = gidx[g];
        const uint16_t code = gcode[g];
        T w[(D == 3) ? 27 : 9];
        ghost_weights<D, T>(code, gw, ng, g, w);
        const int64_t x = pos(X, G.lay);
        r[x] = F[x] - ghost_Bw<D, T>(X, code, w, u, G);
    }
    __syncthreads();
}

// expanded extension of a (the level's r or u) into its band
template <typename T>
__device__ void bt_extend(const BLev<T> &A, T *a) {
    const int64_t nb = A.nb;
    const Lay ly = A.g.lay;
    const uint8_t *const ecnt = A.ecnt;
    const uint32_t *const eg = A.eg, *const bidx = A.bidx;
    const double *const ew = A.ew;
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) {
        EllRound<T> R;
        R.c = 0;
        ell_first<T>(b, ecnt, eg, ew, nb, R);
        a[pos(bidx[b], ly)] = extend_from<T>(b, R, eg, ew, nb, a, ly);
    }
    __syncthreads();
}

// restriction into C from its fine level Fl, the coarse correction zeroed
template <int D, typename T>
__device__ void bt_restrict(const BLev<T> &C, const BLev<T> &Fl) {
    const G2 Gc = C.g, Gf = Fl.g;
    const int64_t nint_c = C.nint, nrow = C.nint + C.ng;
    const T *const rf = Fl.r;
    T *const Fc = C.F, *const Fsc = C.Fs, *const uc = C.u;
    const uint32_t *const ilist = C.ilist, *const gidx = C.gidx, *const fmask = C.fmask;
    for (int64_t row = threadIdx.x; row < nrow; row += blockDim.x) {
        const uint32_t Xc = row < nint_c ? ilist[row] : gidx[row - nint_c];
        int ic[3];
        coords(Xc, (uint32_t)Gc.n, D, ic);
        const T fc = restrict_masked<D, T>(ic, fmask[row], rf, Gf);
        const int64_t xc = pos(Xc, Gc.lay);
        Fc[xc] = fc;
        if (row < nint_c) Fsc[xc] = scaled_rhs<T>(fc, Gc);
        uc[xc] = T(0);
    }
    __syncthreads();
}

// prolongation of C's correction into its fine level Fl
template <int D, typename T>
__device__ void bt_prolong(const BLev<T> &Fl, const BLev<T> &C) {
    const G2 Gf = Fl.g, Gc = C.g;
    const int64_t nint = Fl.nint, nrow = Fl.nint + Fl.ng;
    const T *const ec = C.u;
    T *const uf = Fl.u;
    const uint32_t *const ilist = Fl.ilist, *const gidx = Fl.gidx;
    for (int64_t i = threadIdx.x; i < nrow; i += blockDim.x) {
        const uint32_t X = i < nint ? ilist[i] : gidx[i - nint];
        int iy[3];
        coords(X, (uint32_t)Gf.n, D, iy);
        const int64_t x = pos(X, Gf.lay);
        uf[x] = uf[x] + prolong_at<D, T>(iy, ec, Gc);
    }
    __syncthreads();
}

// coarsest level: u += A^-1 r on the active rows (one warp per row, FP64
// accumulation in the order of kb_coarse_gemv)
template <typename T>
__device__ void bt_coarsest(const BLev<T> &A) {
    const int64_t nact = A.nact;
    const Lay ly = A.g.lay;
    double *const rhs = A.crhs;
    T *const u = A.u;
    const T *const r = A.r;
    const uint32_t *const act = A.act;
    const double *const Ainv = A.Ainv;
    for (int64_t j = threadIdx.x; j < nact; j += blockDim.x) rhs[j] = (double)r[pos(act[j], ly)];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t i = threadIdx.x >> 5; i < nact; i += blockDim.x >> 5) {
        double s = 0.0;
        for (int64_t j = lane; j < nact; j += 32) s = fma(Ainv[i * nact + j], rhs[j], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) u[pos(act[i], ly)] += (T)s;
    }
    __syncthreads();
}

// one block per hierarchy with a tail: its V-cycle from the tail's top
// level down to the coarsest and back (nu1 pre- and nu2 post-smoothing
// steps, each red, black, ghost relaxation)
template <int D, typename T>
__global__ void __launch_bounds__(kBT, 2) kb_btail(const BLev<T> *__restrict__ lv, const BTail *__restrict__ tails,
                                                const BCtl *__restrict__ ctl, int nu1, int nu2) {
    const BTail tl = tails[blockIdx.x];
    const BLev<T> *const L = lv + tl.lev0;
    const int nl = (int)tl.nl;
    if (bskip(ctl, L[0].h)) return;  // uniform over the block (one hierarchy)
    for (int l = 0; l + 1 < nl; ++l) {
        for (int s = 0; s < nu1; ++s) {
            bt_sweep<D, T>(L[l], 0);
            bt_sweep<D, T>(L[l], 1);
            bt_relax<D, T>(L[l]);
        }
        bt_residual<D, T>(L[l]);
        bt_extend<T>(L[l], L[l].r);
        bt_restrict<D, T>(L[l + 1], L[l]);
    }
    bt_residual<D, T>(L[nl - 1]);
    bt_coarsest<T>(L[nl - 1]);
    for (int l = nl - 2; l >= 0; --l) {
        bt_extend<T>(L[l + 1], L[l + 1].u);
        bt_prolong<D, T>(L[l], L[l + 1]);
        for (int s = 0; s < nu2; ++s) {
            bt_sweep<D, T>(L[l], 0);
            bt_sweep<D, T>(L[l], 1);
            bt_relax<D, T>(L[l]);
        }
    }
}

// One block per hierarchy: reduce its norm partials (slots p0[h] .. p0[h+1]
// of the norm residual launch) in slot order, then start (mode 0) or check
// (mode 1) its solve; the last block to finish sets the WHILE condition to
// "more than stop_at hierarchies still run" and resets the counters.
__global__ void __launch_bounds__(256) kb_norm_check(BCtl *__restrict__ ctl, const double *__restrict__ part,
                                                     const int64_t *__restrict__ p0, BShared *sh, int mode,
                                                     unsigned stop_at, cudaGraphConditionalHandle cond) {
    pdl_begin();
    const int h = blockIdx.x;
    __shared__ double red[2][256];
    double a = 0.0, b = 0.0;
    for (int64_t s = p0[h] + threadIdx.x; s < p0[h + 1]; s += blockDim.x) {
        a += part[s * 4 + 0];
        b += part[s * 4 + 1];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            red[0][threadIdx.x] += red[0][threadIdx.x + o];
            red[1][threadIdx.x] += red[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    __shared__ int last;
    if (threadIdx.x == 0) {
        BCtl &c = ctl[h];
        double nrm[2] = {sqrt(red[0][0]), sqrt(red[1][0])};
        const double rn = resid_norm(nrm);
        const bool fin = finite_d(rn);
        if (mode == 0) {
            c.r0 = rn;
            c.cycles = 0;
            c.rel = rn > 0.0 ? 1.0 : 0.0;
            c.status = fin ? BCMG_OK : BCMG_ENONFINITE;
            c.done = !(fin && (rn > 0.0 || c.fixed) && c.max_cycles > 0);
        } else if (!c.done) {
            const int cyc = c.cycles + 1;
            c.cycles = cyc;
            const double rel = c.r0 > 0.0 ? rn / c.r0 : 0.0;
            c.rel = rel;
            if (!fin) c.status = BCMG_ENONFINITE;
            c.done = !(fin && (c.fixed || rel > c.rtol) && cyc < c.max_cycles);
        }
        if (!c.done) atomicAdd(&sh->active, 1u);
        __threadfence();
        last = atomicAdd(&sh->blocks_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const unsigned act = *(volatile unsigned *)&sh->active;
        sh->active = 0u;
        sh->blocks_done = 0u;
        cudaGraphSetConditional(cond, act > stop_at ? 1u : 0u);
    }
}

// ------------------------------------------------------------ host side
template <typename K, typename... A>
void blaunch(cudaStream_t st, K kern, unsigned grid, unsigned block, int64_t *count, A... args) {
    if (grid == 0) return;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    check_cuda(cudaLaunchKernelEx(&cfg, kern, args...), "batched stage");
    ++*count;
}

template <typename T>
BLev<T> blev_of(Handle &H, int l, int h) {
    Level &L = H.L[l];
    BLev<T> b{};
    b.g = g2_of(L);
    b.ilist = L.ilist;
    b.nred = L.nred;
    b.nint = L.nint;
    b.gidx = L.gidx;
    b.gcode = L.gcode;
    b.ng = L.ng;
    b.gdt = L.gdt;
    b.bidx = L.bidx;
    b.ecnt = L.ecnt;
    b.eg = L.eg;
    b.ew = L.ew;
    b.nb = L.nb;
    b.fmask = L.fmask;
    b.act = L.act;
    b.nact = L.nact;
    b.Ainv = L.Ainv;
    b.crhs = L.crhs;
    b.h = h;
    if (sizeof(T) == 8) {
        b.gw = (const T *)L.gw;
        b.u = (T *)(l == 0 ? H.u0 : L.u);
        b.F = (T *)L.F;
        b.Fs = (T *)L.Fs;
        b.r = (T *)L.r;
        b.tmp = (T *)L.gtmp;
    } else {
        b.gw = (const T *)L.gw32;
        b.u = (T *)L.u32;
        b.F = (T *)L.F32;
        b.Fs = (T *)L.Fs32;
        b.r = (T *)L.r32;
        b.tmp = (T *)L.gtmp32;
    }
    return b;
}

// launches of one batch: stage kind, its argument, its ranges and blocks
struct Stage {
    int kind, arg;
    int64_t first, nr, blocks;
    int npt;  // items per thread of the stage's kernel (1 or 4)
};
enum { S_RED, S_BLACK, S_RELAX, S_SCATTER, S_RES, S_EXT_R, S_EXT_U, S_RESTRICT, S_PROLONG, S_GATHER, S_GEMV,
       S_IR_BEGIN, S_IR_UPDATE, S_NORMRES, S_CHECK, S_TAIL };

struct Plan {
    int bs = 128;
    int npt = 1;  // items per thread of the node-parallel stages
    std::vector<BRange> ranges;
    std::vector<BTail> tails;  // block-tail blocks (one per hierarchy with a tail)
    int nu1 = 2, nu2 = 1;
    std::vector<Stage> cycle;  // one cycle (precision of the V-cycle)
    std::vector<Stage> norms;  // finest FP64 residual with partials; refinement rows
    std::vector<int64_t> p0;   // partial slots per hierarchy (norms)
    int64_t nparts = 0;
};

struct Batch {
    std::vector<Handle *> hs;
    int d = 3;
    bool mixed = false;
    std::vector<int> base;  // first level descriptor of each hierarchy
    int nlev = 0;
    std::vector<BLev<double>> l64;
    std::vector<BLev<float>> l32;
};

// the ranges of one stage, n(level) work items per level, per_block items a block
struct StageBuilder {
    Plan &P;
    int64_t first;
    uint32_t blocks = 0;
    int npt;
    explicit StageBuilder(Plan &p, int npt_ = 1) : P(p), first((int64_t)p.ranges.size()), npt(npt_) {}
    template <class Fn>
    void add(const std::vector<int> &levs, int per_block, Fn n_of, uint32_t sub = 0) {
        for (int lv : levs) {
            const int64_t n = n_of(lv);
            const uint32_t nb = (uint32_t)((n + per_block - 1) / per_block);
            if (nb == 0) continue;
            P.ranges.push_back(BRange{(uint32_t)lv, sub, blocks, 0u});
            blocks += nb;
        }
    }
    void push(std::vector<Stage> &seq, int kind, int arg) {
        if (blocks > 0) seq.push_back(Stage{kind, arg, first, (int64_t)P.ranges.size() - first, (int64_t)blocks, npt});
    }
};

// the stages of one cycle and of the norms; node-parallel stages (colour
// sweeps, interior residual rows, restriction and prolongation in 2D, the
// refinement rows) take npt items per thread, the ghost, band and coarsest
// stages one
Plan make_plan(const Batch &B, int bs, int npt, int nu1, int nu2, int64_t tail_rows = 0) {
    Plan P;
    P.bs = bs;
    P.npt = npt;
    P.nu1 = nu1;
    P.nu2 = nu2;
    const int nptr = B.d == 2 ? npt : 1;  // 3^d-point restriction rows: one per thread in 3D
    const int nh = (int)B.hs.size();
    int depth = 0;
    for (Handle *H : B.hs) depth = std::max(depth, (int)H->L.size());
    auto lev = [&](int h, int k) { return B.base[h] + k; };
    auto info = [&](int lv) -> const BLev<double> & { return B.l64[lv]; };
    auto nred = [&](int lv) { return info(lv).nred; };
    auto nblack = [&](int lv) { return info(lv).nint - info(lv).nred; };
    auto nint = [&](int lv) { return info(lv).nint; };
    auto ng = [&](int lv) { return info(lv).ng; };
    auto nrows = [&](int lv) { return info(lv).nint + info(lv).ng; };
    auto nband = [&](int lv) { return info(lv).nb; };
    auto nact = [&](int lv) { return info(lv).nact; };
    // the block tail of each hierarchy: its levels from st[h] down to the
    // coarsest, when every list of each of them has at most tail_rows
    // entries (the coarsest at most kBTMaxCoarse unknowns) and there are at
    // least two; st[h] = L - 1 (no tail) otherwise
    std::vector<int> st(nh);
    std::vector<bool> tailed(nh, false);
    auto fits = [&](int lv) {
        const BLev<double> &A = info(lv);
        const int64_t m = std::max({A.nred, A.nint - A.nred, A.nint + A.ng, A.nb, A.nact});
        return m <= tail_rows && (A.nb == 0 || A.ecnt != nullptr);
    };
    for (int h = 0; h < nh; ++h) {
        const int Lh = (int)B.hs[h]->L.size();
        st[h] = Lh - 1;
        if (tail_rows <= 0 || Lh < 2 || !fits(lev(h, Lh - 1)) || info(lev(h, Lh - 1)).nact > kBTMaxCoarse) continue;
        int t = Lh - 1;
        while (t - 1 >= 1 && fits(lev(h, t - 1))) --t;
        if (t > Lh - 2) continue;
        st[h] = t;
        tailed[h] = true;
        P.tails.push_back(BTail{(uint32_t)lev(h, t), (uint32_t)(Lh - t)});
    }
    std::vector<Stage> &C = P.cycle;
    auto smooth_steps = [&](const std::vector<int> &S, int steps) {
        for (int s = 0; s < steps; ++s) {
            StageBuilder r(P, npt);
            r.add(S, bs * npt, nred);
            r.push(C, S_RED, 0);
            StageBuilder b(P, npt);
            b.add(S, bs * npt, nblack);
            b.push(C, S_BLACK, 1);
            StageBuilder g(P);
            g.add(S, bs, ng);
            g.push(C, S_RELAX, 0);
            StageBuilder c(P);
            c.add(S, bs, ng);
            c.push(C, S_SCATTER, 0);
        }
    };
    // the way down
    for (int k = 0; k < depth; ++k) {
        std::vector<int> S, Co, Sc;
        for (int h = 0; h < nh; ++h) {
            const int Lh = (int)B.hs[h]->L.size();
            if (k < st[h]) {
                S.push_back(lev(h, k));
                Sc.push_back(lev(h, k + 1));
            } else if (k == Lh - 1 && !tailed[h]) {
                Co.push_back(lev(h, k));
            }
        }
        smooth_steps(S, nu1);
        {
            StageBuilder r(P, npt);
            r.add(S, bs * npt, nint, 0);
            r.add(S, bs, ng, 1);
            r.push(C, S_RES, 0);
            StageBuilder e(P);
            e.add(S, bs, nband);
            e.push(C, S_EXT_R, 0);
            StageBuilder q(P, nptr);
            q.add(Sc, bs * nptr, nrows);
            q.push(C, S_RESTRICT, 0);
        }
        if (!Co.empty()) {
            StageBuilder r(P, npt);
            r.add(Co, bs * npt, nint, 0);
            r.add(Co, bs, ng, 1);
            r.push(C, S_RES, 0);
            StageBuilder g(P);
            g.add(Co, bs, nact);
            g.push(C, S_GATHER, 0);
            StageBuilder m(P);
            m.add(Co, bs / 32, nact);
            m.push(C, S_GEMV, 0);
        }
    }
    // the block tails, between the two legs
    if (!P.tails.empty())
        C.push_back(Stage{S_TAIL, 0, 0, (int64_t)P.tails.size(), (int64_t)P.tails.size(), 1});
    // the way up
    for (int k = depth - 2; k >= 0; --k) {
        std::vector<int> S, Cb;
        for (int h = 0; h < nh; ++h)
            if (k < st[h]) {
                S.push_back(lev(h, k));
                Cb.push_back(lev(h, k + 1));
            }
        StageBuilder e(P);
        e.add(Cb, bs, nband);
        e.push(C, S_EXT_U, 1);
        StageBuilder q(P, nptr);
        q.add(S, bs * nptr, nrows);
        q.push(C, S_PROLONG, 0);
        smooth_steps(S, nu2);
    }
    // the finest FP64 residual with norm partials, hierarchy by hierarchy
    // (partial slot = block), then the refinement rows of the finest levels
    {
        StageBuilder r(P, npt);
        P.p0.assign((size_t)nh + 1, 0);
        std::vector<int> L0;
        for (int h = 0; h < nh; ++h) {
            P.p0[h] = r.blocks;
            std::vector<int> one{lev(h, 0)};
            r.add(one, bs * npt, nint, 0);
            r.add(one, bs, ng, 1);
            L0.push_back(lev(h, 0));
        }
        P.p0[nh] = r.blocks;
        P.nparts = r.blocks;
        r.push(P.norms, S_NORMRES, 0);
        StageBuilder ir(P, npt);
        ir.add(L0, bs * npt, nrows);
        ir.push(P.norms, S_IR_BEGIN, 0);
    }
    return P;
}

// device copies of a batch's tables
struct DevPlan {
    BTail *tails = nullptr;
    BLev<double> *l64 = nullptr;
    BLev<float> *l32 = nullptr;
    BRange *ranges = nullptr;
    BCtl *ctl = nullptr;
    BShared *sh = nullptr;
    double *part = nullptr;
    int64_t *p0 = nullptr;
    std::vector<void *> blocks;
};

template <int D, typename T>
void enqueue_stages(const Plan &P, const DevPlan &Dv, const BLev<T> *lv, const std::vector<Stage> &seq,
                    cudaStream_t st, int64_t *count) {
    const unsigned bs = (unsigned)P.bs;
    const BCtl *ctl = Dv.ctl;
    for (const Stage &s : seq) {
        const BRange *rg = Dv.ranges + s.first;
        const int nr = (int)s.nr;
        const unsigned grid = (unsigned)s.blocks;
        switch (s.kind) {
            case S_RED:
            case S_BLACK:
                if (s.npt == 4) blaunch(st, kb_smooth<D, T, 4>, grid, bs, count, lv, rg, nr, ctl, s.arg);
                else blaunch(st, kb_smooth<D, T, 1>, grid, bs, count, lv, rg, nr, ctl, s.arg);
                break;
            case S_RELAX:
                blaunch(st, kb_ghost_relax<D, T>, grid, bs, count, lv, rg, nr, ctl);
                break;
            case S_SCATTER:
                blaunch(st, kb_ghost_scatter<T>, grid, bs, count, lv, rg, nr, ctl);
                break;
            case S_RES:
                if (s.npt == 4) blaunch(st, kb_residual<D, T, 4>, grid, bs, count, lv, rg, nr, ctl, (double *)nullptr);
                else blaunch(st, kb_residual<D, T, 1>, grid, bs, count, lv, rg, nr, ctl, (double *)nullptr);
                break;
            case S_EXT_R:
            case S_EXT_U:
                blaunch(st, kb_extend<T>, grid, bs, count, lv, rg, nr, ctl, s.arg);
                break;
            case S_RESTRICT:
                if constexpr (D == 2)
                    if (s.npt == 4) {
                        blaunch(st, kb_restrict<D, T, 4>, grid, bs, count, lv, rg, nr, ctl);
                        break;
                    }
                blaunch(st, kb_restrict<D, T, 1>, grid, bs, count, lv, rg, nr, ctl);
                break;
            case S_PROLONG:
                if constexpr (D == 2)
                    if (s.npt == 4) {
                        blaunch(st, kb_prolong<D, T, 4>, grid, bs, count, lv, rg, nr, ctl);
                        break;
                    }
                blaunch(st, kb_prolong<D, T, 1>, grid, bs, count, lv, rg, nr, ctl);
                break;
            case S_GATHER:
                blaunch(st, kb_coarse_gather<T>, grid, bs, count, lv, rg, nr, ctl);
                break;
            case S_GEMV:
                blaunch(st, kb_coarse_gemv<T>, grid, bs, count, lv, rg, nr, ctl);
                break;
            case S_TAIL:
                blaunch(st, kb_btail<D, T>, grid, (unsigned)kBT, count, lv, (const BTail *)Dv.tails, ctl, P.nu1,
                        P.nu2);
                break;
            default:
                break;
        }
    }
}

// the finest FP64 residual with partials, then the check (mode 0 start, 1
// per cycle)
template <int D>
void enqueue_norms(const Batch &B, const Plan &P, const DevPlan &Dv, cudaStream_t st, int mode, unsigned stop_at,
                   cudaGraphConditionalHandle cond, int64_t *count) {
    const Stage &s = P.norms[0];
    auto kern = s.npt == 4 ? kb_residual<D, double, 4> : kb_residual<D, double, 1>;
    blaunch(st, kern, (unsigned)s.blocks, (unsigned)P.bs, count, (const BLev<double> *)Dv.l64,
            (const BRange *)(Dv.ranges + s.first), (int)s.nr, (const BCtl *)Dv.ctl, Dv.part);
    blaunch(st, kb_norm_check, (unsigned)B.hs.size(), 256u, count, Dv.ctl, (const double *)Dv.part,
            (const int64_t *)Dv.p0, Dv.sh, mode, stop_at, cond);
}

template <int D>
void enqueue_cycle(const Batch &B, const Plan &P, const DevPlan &Dv, cudaStream_t st, int64_t *count) {
    if (!B.mixed) {
        enqueue_stages<D, double>(P, Dv, Dv.l64, P.cycle, st, count);
        return;
    }
    const Stage &ir = P.norms[1];
    const BRange *rg = Dv.ranges + ir.first;
    const bool four = ir.npt == 4;
    blaunch(st, four ? kb_ir_begin<4> : kb_ir_begin<1>, (unsigned)ir.blocks, (unsigned)P.bs, count,
            (const BLev<double> *)Dv.l64, (const BLev<float> *)Dv.l32, rg, (int)ir.nr, (const BCtl *)Dv.ctl);
    enqueue_stages<D, float>(P, Dv, Dv.l32, P.cycle, st, count);
    blaunch(st, four ? kb_ir_update<4> : kb_ir_update<1>, (unsigned)ir.blocks, (unsigned)P.bs, count,
            (const BLev<double> *)Dv.l64, (const BLev<float> *)Dv.l32, rg, (int)ir.nr, (const BCtl *)Dv.ctl);
}

void *dev_alloc(DevPlan &Dv, size_t bytes, cudaStream_t st) {
    void *p = nullptr;
    check_cuda(cudaMallocAsync(&p, std::max<size_t>(bytes, 16), st), "batch tables");
    Dv.blocks.push_back(p);
    return p;
}

template <class V>
void upload(const V &v, void *dst, cudaStream_t st) {
    if (!v.empty())
        check_cuda(cudaMemcpyAsync(dst, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice, st),
                   "batch upload");
}

DevPlan upload_plan(const Batch &B, const Plan &P, cudaStream_t st) {
    DevPlan Dv;
    Dv.l64 = (BLev<double> *)dev_alloc(Dv, sizeof(BLev<double>) * B.l64.size(), st);
    upload(B.l64, Dv.l64, st);
    if (B.mixed) {
        Dv.l32 = (BLev<float> *)dev_alloc(Dv, sizeof(BLev<float>) * B.l32.size(), st);
        upload(B.l32, Dv.l32, st);
    }
    Dv.ranges = (BRange *)dev_alloc(Dv, sizeof(BRange) * P.ranges.size(), st);
    upload(P.ranges, Dv.ranges, st);
    Dv.tails = (BTail *)dev_alloc(Dv, sizeof(BTail) * std::max<size_t>(P.tails.size(), 1), st);
    upload(P.tails, Dv.tails, st);
    Dv.ctl = (BCtl *)dev_alloc(Dv, sizeof(BCtl) * B.hs.size(), st);
    Dv.sh = (BShared *)dev_alloc(Dv, sizeof(BShared), st);
    check_cuda(cudaMemsetAsync(Dv.sh, 0, sizeof(BShared), st), "batch counters");
    Dv.part = (double *)dev_alloc(Dv, sizeof(double) * 4 * (size_t)std::max<int64_t>(P.nparts, 1), st);
    Dv.p0 = (int64_t *)dev_alloc(Dv, sizeof(int64_t) * P.p0.size(), st);
    upload(P.p0, Dv.p0, st);
    return Dv;
}

void free_plan(DevPlan &Dv, cudaStream_t st) {
    for (void *p : Dv.blocks) cudaFreeAsync(p, st);
    Dv.blocks.clear();
}

// one round of the batched solve as one graph: (with start) the start
// norms, then WHILE (cycle, norms, check) while more than stop_at
// hierarchies run; without start the loop is entered directly (the states
// carry on from an earlier round)
template <int D>
cudaGraphExec_t build_batch_graph(const Batch &B, const Plan &P, const DevPlan &Dv, cudaStream_t st, bool start,
                                  unsigned stop_at, int64_t *prefix, int64_t *body) {
    cudaGraph_t g = nullptr;
    check_cuda(cudaGraphCreate(&g, 0), "cudaGraphCreate");
    cudaGraphConditionalHandle cond;
    check_cuda(cudaGraphConditionalHandleCreate(&cond, g, start ? 0u : 1u, cudaGraphCondAssignDefault),
               "conditional handle");
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    *prefix = 0;
    if (start) {
        check_cuda(cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                   "capture batch prefix");
        enqueue_norms<D>(B, P, Dv, st, 0, stop_at, cond, prefix);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        check_cuda(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd), "capture info");
        cudaGraphNode_t cn;
        check_cuda(cudaGraphAddNode(&cn, g, deps, nullptr, nd, &p), "WHILE node");
        check_cuda(cudaStreamUpdateCaptureDependencies(st, &cn, nullptr, 1, cudaStreamSetCaptureDependencies),
                   "capture dependencies");
        check_cuda(cudaStreamEndCapture(st, &g), "end capture prefix");
    } else {
        cudaGraphNode_t cn;
        check_cuda(cudaGraphAddNode(&cn, g, nullptr, nullptr, 0, &p), "WHILE node");
    }
    cudaGraph_t bodyg = p.conditional.phGraph_out[0];
    check_cuda(cudaStreamBeginCaptureToGraph(st, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
               "capture batch body");
    *body = 0;
    enqueue_cycle<D>(B, P, Dv, st, body);
    enqueue_norms<D>(B, P, Dv, st, 1, stop_at, cond, body);
    check_cuda(cudaStreamEndCapture(st, &bodyg), "end capture body");
    cudaGraphExec_t ex = nullptr;
    check_cuda(cudaGraphInstantiate(&ex, g, 0), "instantiate batch graph");
    cudaGraphDestroy(g);
    return ex;
}

// one batched cycle, captured (for the block-size measurement)
template <int D>
cudaGraphExec_t build_cycle_graph(const Batch &B, const Plan &P, const DevPlan &Dv, cudaStream_t st) {
    cudaGraph_t g = nullptr;
    check_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "capture batch cycle");
    int64_t n = 0;
    enqueue_cycle<D>(B, P, Dv, st, &n);
    check_cuda(cudaStreamEndCapture(st, &g), "end capture cycle");
    cudaGraphExec_t ex = nullptr;
    check_cuda(cudaGraphInstantiate(&ex, g, 0), "instantiate cycle graph");
    cudaGraphDestroy(g);
    return ex;
}

std::mutex g_tune_mu;
std::tuple<int, int, int64_t> g_shape_override{0, 1, 0};  // block 0: none (guarded by g_tune_mu)
std::tuple<int, int, int64_t> g_last_shape{0, 1, 0};      // of the last batched solve (g_tune_mu)
// (dev, d, mixed, nh, nodes) -> (block size, items per thread, tail rows)
std::map<std::tuple<int, int, int, int64_t, int64_t>, std::tuple<int, int, int64_t>> g_tuned;

Batch make_batch(const std::vector<Handle *> &hs) {
    Batch B;
    B.hs = hs;
    B.d = hs[0]->d;
    B.mixed = hs[0]->o.precision == BCMG_PREC_MIXED;
    for (size_t h = 0; h < hs.size(); ++h) {
        B.base.push_back(B.nlev);
        for (int l = 0; l < (int)hs[h]->L.size(); ++l) {
            B.l64.push_back(blev_of<double>(*hs[h], l, (int)h));
            if (B.mixed) B.l32.push_back(blev_of<float>(*hs[h], l, (int)h));
        }
        B.nlev += (int)hs[h]->L.size();
    }
    return B;
}

constexpr int kTuneReplays = 3;       // timed replays per candidate (the fastest counts)
constexpr float kTailSlack = 1.03f;   // the block tail is kept within 3 % of the fastest stage-only shape

// A batch's launch shape: block size and items per thread of the stages,
// and the largest list of a level that runs in the block tail (0: no tail)
struct Shape {
    int bs = 0, npt = 1;
    int64_t tail = 0;
};

// the autotuner: one batched cycle per candidate launch shape, timed after a
// warm replay, on the working copies (saved before and restored after).
// First block size 64, 128 or 256 threads, each with one or four items per
// thread in the node-parallel stages; then, with the fastest of those, the
// block tail for levels of at most 512 or 2048 list entries (the faster of
// the two), kept unless slower than kTailSlack times the stage-only shape.
Shape tune_launch_shape(const Batch &B, cudaStream_t st, double rtol, int max_cycles, int64_t *launched) {
    const int nu1 = B.hs[0]->o.nu1, nu2 = B.hs[0]->o.nu2;
    std::vector<double *> saved;
    for (Handle *H : B.hs) {
        double *p = nullptr;
        const size_t bytes = sizeof(double) * split_len(H->L[0].nn);
        check_cuda(cudaMallocAsync(&p, bytes, st), "tune save");
        check_cuda(cudaMemcpyAsync(p, H->u0, bytes, cudaMemcpyDeviceToDevice, st), "tune save copy");
        saved.push_back(p);
    }
    // the second replay's time; < 0 when the shape gives the batch no tail
    auto time_shape = [&](const Shape &c) -> float {
        Plan P = make_plan(B, c.bs, c.npt, nu1, nu2, c.tail);
        if (c.tail > 0 && P.tails.empty()) return -1.0f;
        DevPlan Dv = upload_plan(B, P, st);
        std::vector<BCtl> c0(B.hs.size());
        for (auto &x : c0) x = BCtl{rtol, max_cycles, 0, 1.0, 1.0, 0, 0, 0};
        upload(c0, Dv.ctl, st);
        cudaGraphExec_t ex = B.d == 3 ? build_cycle_graph<3>(B, P, Dv, st) : build_cycle_graph<2>(B, P, Dv, st);
        cudaEvent_t e0, e1;
        check_cuda(cudaEventCreate(&e0), "event");
        check_cuda(cudaEventCreate(&e1), "event");
        check_cuda(cudaGraphLaunch(ex, st), "tune warm");
        float ms = 0.0f;
        for (int rep = 0; rep < kTuneReplays; ++rep) {
            check_cuda(cudaEventRecord(e0, st), "event");
            check_cuda(cudaGraphLaunch(ex, st), "tune timed");
            check_cuda(cudaEventRecord(e1, st), "event");
            check_cuda(cudaEventSynchronize(e1), "tune sync");
            float t = 0.0f;
            check_cuda(cudaEventElapsedTime(&t, e0, e1), "event time");
            ms = rep == 0 ? t : std::min(ms, t);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaGraphExecDestroy(ex);
        free_plan(Dv, st);
        *launched += (1 + kTuneReplays) * (int64_t)(P.cycle.size() + (B.mixed ? 2 : 0));
        return ms;
    };
    Shape best;
    float best_ms = 0.0f;
    for (const auto cand : {std::make_pair(64, 1), std::make_pair(128, 1), std::make_pair(256, 1),
                            std::make_pair(64, 4), std::make_pair(128, 4), std::make_pair(256, 4)}) {
        const Shape c{cand.first, cand.second, 0};
        const float ms = time_shape(c);
        if (best.bs == 0 || ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    // the replay runs every hierarchy; later rounds run few, where a cycle is
    // bound by its launches, which the tail removes: the tail is kept unless
    // it is measurably slower on the full batch
    const Shape base = best;
    const float base_ms = best_ms;
    float tail_ms = 0.0f;
    for (const int64_t tail : {(int64_t)512, (int64_t)2048}) {
        const Shape c{base.bs, base.npt, tail};
        const float ms = time_shape(c);
        if (ms >= 0.0f && ms <= base_ms * kTailSlack && (best.tail == 0 || ms < tail_ms)) {
            tail_ms = ms;
            best = c;
        }
    }
    for (size_t h = 0; h < B.hs.size(); ++h) {
        check_cuda(cudaMemcpyAsync(B.hs[h]->u0, saved[h], sizeof(double) * split_len(B.hs[h]->L[0].nn),
                                   cudaMemcpyDeviceToDevice, st),
                   "tune restore");
        cudaFreeAsync(saved[h], st);
    }
    return best;
}

}  // namespace

namespace {
// a handle's part of a batched copy of the caller's u in or out
struct BCopy {
    const uint32_t *ilist, *gidx, *box;
    int64_t nint, ng, nbox;
    const double *src;
    double *dst;
    Lay lay;
    uint32_t blk0;  // first block of this handle
};

// in (to_split): the caller's dense u of interior, ghost and eliminated box
// nodes into the working copy; out: interior and ghost nodes back (the
// per-handle copy_active, for every handle of the batch in one launch)
__global__ void __launch_bounds__(256) kb_copy_active(const BCopy *__restrict__ tab, int n, int to_split) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].blk0 <= blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const BCopy &c = tab[lo];
    const int64_t i = (int64_t)(blockIdx.x - c.blk0) * blockDim.x + threadIdx.x;
    const int64_t nbox = to_split ? c.nbox : 0;
    if (i >= c.nint + c.ng + nbox) return;
    int64_t X;
    if (i < c.nint) X = c.ilist[i];
    else if (i < c.nint + c.ng) X = c.gidx[i - c.nint];
    else X = c.box[i - c.nint - c.ng];
    if (to_split) c.dst[pos(X, c.lay)] = c.src[X];
    else c.dst[X] = c.src[pos(X, c.lay)];
}
}  // namespace

// every handle's u between the caller's arrays and the working copies, one
// launch on st (the table goes up with one copy)
void batch_copy_active(const std::vector<Handle *> &hs, double *const *u_devs, cudaStream_t st, bool in) {
    std::vector<BCopy> tab;
    uint32_t blocks = 0;
    for (size_t i = 0; i < hs.size(); ++i) {
        Handle &H = *hs[i];
        const Level &L = H.L[0];
        BCopy c;
        c.ilist = L.ilist;
        c.gidx = L.gidx;
        c.box = L.boxidx;
        c.nint = L.nint;
        c.ng = L.ng;
        c.nbox = L.nbox;
        c.src = in ? u_devs[i] : H.u0;
        c.dst = in ? H.u0 : u_devs[i];
        c.lay = L.lay;
        c.blk0 = blocks;
        tab.push_back(c);
        blocks += (uint32_t)((L.nint + L.ng + (in ? L.nbox : 0) + 255) / 256);
    }
    if (blocks == 0) return;
    BCopy *tab_d = nullptr;
    check_cuda(cudaMallocAsync(&tab_d, sizeof(BCopy) * tab.size(), st), "batch copy table");
    check_cuda(cudaMemcpyAsync(tab_d, tab.data(), sizeof(BCopy) * tab.size(), cudaMemcpyHostToDevice, st),
               "batch copy table");
    kb_copy_active<<<blocks, 256, 0, st>>>(tab_d, (int)tab.size(), in ? 1 : 0);
    check_cuda(cudaGetLastError(), "batch copy");
    add_launches(1);
    cudaFreeAsync(tab_d, st);
}

void batch_last_shape(int *block, int *items, int64_t *tail_rows) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    *block = std::get<0>(g_last_shape);
    *items = std::get<1>(g_last_shape);
    *tail_rows = std::get<2>(g_last_shape);
}

void batch_shape_override(int block, int items, int64_t tail_rows) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_shape_override = std::make_tuple(block, items, tail_rows);
}

bool batch_eligible(const std::vector<Handle *> &hs) {
    if (hs.size() < 2) return false;
    const Handle &H0 = *hs[0];
    for (Handle *H : hs) {
        if (H->d != H0.d || H->o.precision != H0.o.precision || H->o.ordering != BCMG_ORDER_RB ||
            H->o.cycle != BCMG_CYCLE_V || H->o.nu1 != H0.o.nu1 || H->o.nu2 != H0.o.nu2 || H->dev != H0.dev)
            return false;
        for (auto &L : H->L)
            if (L.nb > 0 && !L.ecnt) return false;
    }
    return true;
}

// Solve every hierarchy of hs (eligible batch) from its working copy u0
// (already copied in, ordered on st); per-hierarchy results into the host
// arrays.  The solve runs in rounds: a round's loop stops once at most an
// eighth of its hierarchies still run, and the next round is planned for
// those only, so hierarchies that need many more cycles than the rest (or
// never converge) do not keep every launch of the batch going.  With fixed,
// every hierarchy runs exactly max_cycles cycles (batched V-cycles; only a
// non-finite norm stops one early).  Returns the number of kernels launched.
int64_t batch_solve(const std::vector<Handle *> &hs, cudaStream_t st, double rtol, int max_cycles, int *cycles,
                    double *rels, int *statuses, bool fixed) {
    const int n = (int)hs.size();
    int64_t nodes = 0;
    for (Handle *H : hs)
        for (auto &L : H->L) nodes += L.nint + L.ng;
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    // batches of similar size share a tuned shape: the count of hierarchies
    // and their rows are keyed rounded up to powers of two (a stream of
    // batches that all differ, as a server forms them, is tuned once per
    // size class, not once per batch)
    auto pow2 = [](int64_t v) {
        int64_t p = 1;
        while (p < v) p <<= 1;
        return p;
    };
    const auto key =
        std::make_tuple(dev, hs[0]->d, (int)(hs[0]->o.precision == BCMG_PREC_MIXED), pow2(n), pow2(nodes));
    int64_t launched = 0;
    Shape shape;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (std::get<0>(g_shape_override) > 0)
            shape = Shape{std::get<0>(g_shape_override), std::get<1>(g_shape_override),
                          std::get<2>(g_shape_override)};
        auto it = g_tuned.find(key);
        if (shape.bs == 0 && it != g_tuned.end())
            shape = Shape{std::get<0>(it->second), std::get<1>(it->second), std::get<2>(it->second)};
    }
    if (shape.bs == 0) {
        shape = tune_launch_shape(make_batch(hs), st, rtol, max_cycles, &launched);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = std::make_tuple(shape.bs, shape.npt, shape.tail);
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_last_shape = std::make_tuple(shape.bs, shape.npt, shape.tail);
    }
    std::vector<BCtl> state(n, BCtl{rtol, max_cycles, 0, 0.0, 0.0, 0, 0, fixed ? 1 : 0});
    std::vector<int> active(n);
    for (int i = 0; i < n; ++i) active[i] = i;
    bool start = true;
    while (!active.empty()) {
        std::vector<Handle *> sub;
        std::vector<BCtl> cs;
        for (int i : active) {
            sub.push_back(hs[i]);
            cs.push_back(state[i]);
        }
        const Batch B = make_batch(sub);
        const Plan P = make_plan(B, shape.bs, shape.npt, hs[0]->o.nu1, hs[0]->o.nu2, shape.tail);
        DevPlan Dv = upload_plan(B, P, st);
        upload(cs, Dv.ctl, st);
        const unsigned stop_at = active.size() > 8 ? (unsigned)(active.size() / 8) : 0u;
        int64_t prefix = 0, body = 0;
        cudaGraphExec_t ex = B.d == 3 ? build_batch_graph<3>(B, P, Dv, st, start, stop_at, &prefix, &body)
                                      : build_batch_graph<2>(B, P, Dv, st, start, stop_at, &prefix, &body);
        check_cuda(cudaGraphLaunch(ex, st), "batch solve");
        check_cuda(cudaMemcpyAsync(cs.data(), Dv.ctl, sizeof(BCtl) * cs.size(), cudaMemcpyDeviceToHost, st),
                   "batch state");
        check_cuda(cudaStreamSynchronize(st), "batch sync");
        cudaGraphExecDestroy(ex);
        free_plan(Dv, st);
        int ran = 0;
        std::vector<int> next;
        for (size_t j = 0; j < active.size(); ++j) {
            ran = std::max(ran, cs[j].cycles - state[active[j]].cycles);
            state[active[j]] = cs[j];
            if (!cs[j].done) next.push_back(active[j]);
        }
        launched += prefix + body * (int64_t)ran;
        if (next.size() == active.size() && ran == 0) break;  // no progress (cannot happen; a guard)
        active.swap(next);
        start = false;
    }
    for (int i = 0; i < n; ++i) {
        const BCtl &c = state[i];
        cycles[i] = c.cycles;
        rels[i] = c.rel;
        int status = c.status;
        if (!fixed && status == BCMG_OK && c.r0 > 0.0 && c.rel > rtol) status = BCMG_ENOCONV;
        statuses[i] = status;
    }
    return launched;
}

}  // namespace bcmg
