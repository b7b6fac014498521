// Multigrid cycle kernels of the GB300 BCMG library (arXiv 2207.14208).
//
// Interior work runs over compacted per-colour lists of interior nodes (red
// then black, increasing index), so every lane of a warp does useful work:
// on GB300 the FP64 pipe executes whole warp instructions, so idle lanes
// would cost FP64 throughput.  Ghost and band work runs over their compacted
// lists.  Every cycle kernel is templated on the value type: FP64 for the
// plain cycle, FP32 for the inner cycle of the mixed-precision refinement.
// GB300 executes FP64 at 2 FMA per clock per SM, so FP64 work is spread over
// all SMs (block sizes shrink on small levels) and kept short (the ghost
// interpolation weights are tabulated once).  The coarse end of the V-cycle
// runs as one kernel on a thread-block cluster, its phases separated by the
// hardware cluster barrier.  None of these kernels is a dense contraction,
// so no tensor-core path is used.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "bcmg_internal.cuh"
#include "nodeops.cuh"

namespace bcmg {

namespace {

// ------------------------------------------------------------ grid kernels
template <int D, typename T>
// Fs != null: the update from the scaled right-hand side (the cycle's
// levels keep it); else from F (a caller's own F).  par 0 / 1: every node of
// the list has that index parity and n is odd; -1: no such promise
__global__ void __launch_bounds__(kT) k_smooth(const uint32_t *__restrict__ list, int64_t n, T *u,
                                               const T *__restrict__ F, const T *__restrict__ Fs, G2 G, int par) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t X = i < n ? list[i] : 0u;
    pdl_begin();
    if (i < n) {
        if (Fs && par >= 0) smooth_at_par<D, T>(X, u, Fs, G, par);
        else if (Fs) smooth_at_s<D, T>(X, u, Fs, G);
        else smooth_at<D, T>(X, u, F, G);
    }
}

// The colour sweep of a large FP32 level on a parity-split level with odd n,
// as a persistent grid: the SMs' resident blocks walk the list in chunks of
// NPT x blockDim entries (chunks blockIdx, blockIdx + gridDim, ...; entry
// i0 + j blockDim, coalesced per j).  A thread's NPT entries' loads are all
// issued before any update, and the list entries of its next chunk are
// loaded while the values of the current one are in flight, so past its
// first chunk a block waits for one round trip per chunk, not two (the sweep
// is bound by memory latency, not by arithmetic).  A colour sweep reads only
// the other colour and writes only its own, so no entry depends on another.
// Same terms, same order as smooth_at_par.
template <int D, typename T, int NPT>
__global__ void __launch_bounds__(kT) k_smooth_pers(const uint32_t *__restrict__ list, int64_t n, T *u,
                                                    const T *__restrict__ Fs, G2 G, int par) {
    const int64_t chunk = (int64_t)blockDim.x * NPT;
    int64_t c = blockIdx.x;
    uint32_t m[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t i = c * chunk + (int64_t)j * blockDim.x + threadIdx.x;
        m[j] = i < n ? (list[i] >> 1) : 0u;
    }
    pdl_begin();
    const int64_t sy = G.sy, sz = G.sz;
    const int64_t xm = par - 1, xp = par, ym = par - ((sy + 1) >> 1), yp = par + ((sy - 1) >> 1);
    const int64_t zm = par - ((sz + 1) >> 1), zp = par + ((sz - 1) >> 1);
    const T *v = u + (par ? 0 : G.lay.ho);
    const int64_t own = par ? G.lay.ho : 0;
    for (; c * chunk < n; c += gridDim.x) {
        const int64_t i0 = c * chunk + threadIdx.x;
        T a[NPT][D == 3 ? 6 : 4], f[NPT];
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const bool on = i0 + (int64_t)j * blockDim.x < n;
            const T *w = v + m[j];
            a[j][0] = on ? w[xm] : T(0);
            a[j][1] = on ? w[xp] : T(0);
            a[j][2] = on ? w[ym] : T(0);
            a[j][3] = on ? w[yp] : T(0);
            if (D == 3) {
                a[j][4] = on ? w[zm] : T(0);
                a[j][5] = on ? w[zp] : T(0);
            }
            f[j] = on ? Fs[own + m[j]] : T(0);
        }
        uint32_t mn[NPT];
        const int64_t i1 = (c + gridDim.x) * chunk + threadIdx.x;
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const int64_t i = i1 + (int64_t)j * blockDim.x;
            mn[j] = i < n ? (list[i] >> 1) : 0u;
        }
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            if (i0 + (int64_t)j * blockDim.x >= n) continue;
            T s = (a[j][0] + a[j][1]) + (a[j][2] + a[j][3]);
            if (D == 3) s += a[j][4] + a[j][5];
            u[own + m[j]] = fma(s, (T)G.inv_diag, f[j]);
        }
#pragma unroll
        for (int j = 0; j < NPT; ++j) m[j] = mn[j];
    }
}

// k_smooth_pers with 16-bit storage: u and Fs held as bfloat16 (8-bit
// significand), every sum and the update in FP32, the new value rounded to
// bfloat16 (round to nearest even).  Used only to measure what 16-bit
// storage would gain on the dominant kernel (time_sweeps_bf16).
template <int D, int NPT>
__global__ void __launch_bounds__(kT) k_smooth_pers_bf16(const uint32_t *__restrict__ list, int64_t n,
                                                         __nv_bfloat16 *u, const __nv_bfloat16 *__restrict__ Fs,
                                                         G2 G, int par) {
    const int64_t chunk = (int64_t)blockDim.x * NPT;
    int64_t c = blockIdx.x;
    uint32_t m[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t i = c * chunk + (int64_t)j * blockDim.x + threadIdx.x;
        m[j] = i < n ? (list[i] >> 1) : 0u;
    }
    pdl_begin();
    const int64_t sy = G.sy, sz = G.sz;
    const int64_t xm = par - 1, xp = par, ym = par - ((sy + 1) >> 1), yp = par + ((sy - 1) >> 1);
    const int64_t zm = par - ((sz + 1) >> 1), zp = par + ((sz - 1) >> 1);
    const __nv_bfloat16 *v = u + (par ? 0 : G.lay.ho);
    const int64_t own = par ? G.lay.ho : 0;
    const float inv_diag = (float)G.inv_diag;
    for (; c * chunk < n; c += gridDim.x) {
        const int64_t i0 = c * chunk + threadIdx.x;
        float a[NPT][D == 3 ? 6 : 4], f[NPT];
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const bool on = i0 + (int64_t)j * blockDim.x < n;
            const __nv_bfloat16 *w = v + m[j];
            a[j][0] = on ? __bfloat162float(w[xm]) : 0.0f;
            a[j][1] = on ? __bfloat162float(w[xp]) : 0.0f;
            a[j][2] = on ? __bfloat162float(w[ym]) : 0.0f;
            a[j][3] = on ? __bfloat162float(w[yp]) : 0.0f;
            if (D == 3) {
                a[j][4] = on ? __bfloat162float(w[zm]) : 0.0f;
                a[j][5] = on ? __bfloat162float(w[zp]) : 0.0f;
            }
            f[j] = on ? __bfloat162float(Fs[own + m[j]]) : 0.0f;
        }
        uint32_t mn[NPT];
        const int64_t i1 = (c + gridDim.x) * chunk + threadIdx.x;
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const int64_t i = i1 + (int64_t)j * blockDim.x;
            mn[j] = i < n ? (list[i] >> 1) : 0u;
        }
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            if (i0 + (int64_t)j * blockDim.x >= n) continue;
            float s = (a[j][0] + a[j][1]) + (a[j][2] + a[j][3]);
            if (D == 3) s += a[j][4] + a[j][5];
            u[own + m[j]] = __float2bfloat16_rn(fmaf(s, inv_diag, f[j]));
        }
#pragma unroll
        for (int j = 0; j < NPT; ++j) m[j] = mn[j];
    }
}

template <typename S>
__global__ void k_to_bf16(const S *__restrict__ src, __nv_bfloat16 *__restrict__ dst, int64_t n) {
    pdl_begin();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn((float)src[i]);
}

// fictitious-time relaxation of every ghost from the same u (eq. rel with
// eq. DtauOptTheta): tmp_g = u_G + dt_g (g_G - B u~); k_ghost_scatter writes
// tmp back once all ghosts are done (Jacobi over the ghosts)
template <int D, typename T>
__global__ void __launch_bounds__(kT) k_ghost_relax(const uint32_t *__restrict__ gidx,
                                                    const uint16_t *__restrict__ gcode, const T *__restrict__ gw,
                                                    const double *__restrict__ gdt, int64_t ng, const T *u,
                                                    const T *__restrict__ F, T *__restrict__ tmp, G2 G) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = g < ng;
    const int64_t X = on ? gidx[g] : 0;
    const uint16_t code = on ? gcode[g] : 0;
    const T dt = on ? (T)gdt[g] : T(0);
    T w[(D == 3) ? 27 : 9];
    ghost_weights<D, T>(code, gw, ng, on ? g : 0, w);
    pdl_begin();
    if (on) {
        const int64_t x = pos(X, G.lay);
        tmp[g] = fma(dt, F[x] - ghost_Bw<D, T>(X, code, w, u, G), u[x]);
    }
}

template <typename T>
__global__ void __launch_bounds__(kT) k_ghost_scatter(const uint32_t *__restrict__ gidx, int64_t ng,
                                                      const T *__restrict__ tmp, T *__restrict__ u, Lay ly) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t X = g < ng ? gidx[g] : 0u;
    pdl_begin();
    if (g < ng) u[pos(X, ly)] = tmp[g];
}

// ------------------------------------------------------------ solve control
// before the loop: r0 from the initial norms; run the body iff r0 > 0 is
// finite and cycles are allowed
__device__ void solve_init_dev(SolveState *st, const double *nout, cudaGraphConditionalHandle cond) {
    const double r0 = resid_norm(nout);
    const bool fin = finite_d(r0);
    st->r0 = r0;
    st->cycles = 0;
    st->rel = r0 > 0.0 ? 1.0 : 0.0;
    st->status = fin ? BCMG_OK : BCMG_ENONFINITE;
    cudaGraphSetConditional(cond, (fin && r0 > 0.0 && st->max_cycles > 0) ? 1u : 0u);
}

// after each cycle: count it, relative residual, continue while above rtol
__device__ void solve_check_dev(SolveState *st, const double *nout, cudaGraphConditionalHandle cond) {
    const int c = st->cycles + 1;
    st->cycles = c;
    const double rn = resid_norm(nout);
    const double rel = rn / st->r0;
    st->rel = rel;
    const bool fin = finite_d(rn);
    if (!fin) st->status = BCMG_ENONFINITE;
    cudaGraphSetConditional(cond, (fin && rel > st->rtol && c < st->max_cycles) ? 1u : 0u);
}

// What the last block of the ghost residual kernel does once every partial
// is written: mode 1 the four norms into nout, mode 2 also the solve's start
// (solve_init_dev), mode 3 also the per-cycle check (solve_check_dev).
struct NormTail {
    int mode;
    int64_t nparts;     // partials of the interior and the ghost kernels
    unsigned *counter;  // ghost blocks done (zero between uses)
    double *nout;
    SolveState *st;
    cudaGraphConditionalHandle cond;
};

// the last-arriving block (fence, then a counter) reduces all partials in
// block order, like k_norm_final, and resets the counter
template <bool Ctl>
__device__ void norm_tail(const NormTail &nt, const double *part) {
    __shared__ int last;
    __shared__ double sh[4][kT / 32];
    __syncthreads();  // this block's partial is written
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(nt.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;  // uniform over the block
    __threadfence();
    // eight partials per thread in flight at once (16-byte loads), then
    // folded in slot order
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    const double2 *p2 = reinterpret_cast<const double2 *>(part);
    constexpr int U = 8;
    for (int64_t i0 = threadIdx.x; i0 < nt.nparts; i0 += (int64_t)U * blockDim.x) {
        double2 lo[U], hi[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x;
            const bool ok = i < nt.nparts;
            lo[u] = ok ? __ldcg(p2 + 2 * i) : make_double2(0.0, 0.0);
            hi[u] = ok ? __ldcg(p2 + 2 * i + 1) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            a[0] += lo[u].x;
            a[1] += lo[u].y;
            a[2] = fmax(a[2], hi[u].x);
            a[3] = fmax(a[3], hi[u].y);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a[0] += __shfl_down_sync(0xffffffffu, a[0], o);
        a[1] += __shfl_down_sync(0xffffffffu, a[1], o);
        a[2] = fmax(a[2], __shfl_down_sync(0xffffffffu, a[2], o));
        a[3] = fmax(a[3], __shfl_down_sync(0xffffffffu, a[3], o));
    }
    if (lane == 0)
        for (int q = 0; q < 4; ++q) sh[q][warp] = a[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        double b[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < nw; ++w) {
            b[0] += sh[0][w];
            b[1] += sh[1][w];
            b[2] = fmax(b[2], sh[2][w]);
            b[3] = fmax(b[3], sh[3][w]);
        }
        nt.nout[0] = sqrt(b[0]);
        nt.nout[1] = sqrt(b[1]);
        nt.nout[2] = b[2];
        nt.nout[3] = b[3];
        *nt.counter = 0u;
        if constexpr (Ctl) {
            if (nt.mode == 2) solve_init_dev(nt.st, nt.nout, nt.cond);
            else if (nt.mode == 3) solve_check_dev(nt.st, nt.nout, nt.cond);
        }
    }
}

// r = F - A u on the interior rows (eq. Laph); with part != null also the
// block's norm partials (slot = block).  NPT rows per thread (strided by the
// block size): with norm partials the squares are summed in the thread first
// (one FMA per row), so the warp reduction's FP64 adds are shared by NPT rows.
// With after != 0 (right after a red-black smoothing step of the level) the
// black rows whose neighbours are all interior are not computed: the black
// sweep solved their equations from the red values and the ghost relaxation
// after it changed no neighbour of theirs, so their residual is zero (up to
// the sweep's rounding) and is stored as such, with no loads and no
// arithmetic.  The other black rows (bit set in bmask) are computed from
// their own sorted list bnear, in the grid's first nbn rows (their loads are
// scattered along the boundary: started first, they overlap the rest).
template <int D, typename T, int NPT>
__global__ void __launch_bounds__(kT) k_residual_int(const uint32_t *__restrict__ ilist, int64_t nint, int64_t nred,
                                                     const uint32_t *__restrict__ bmask,
                                                     const uint32_t *__restrict__ bnear, int64_t nbn, int after,
                                                     const T *__restrict__ u, const T *__restrict__ F,
                                                     T *__restrict__ r, G2 G, double *__restrict__ part) {
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x * NPT + threadIdx.x;
    const int64_t rows = after ? nint + nbn : nint;
    int64_t X[NPT];
    int mode[NPT];  // 0 nothing, 1 computed, 2 zero
    const int64_t head = after ? nbn : 0;  // rows of bnear before the list's
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int64_t i = i0 + (int64_t)j * blockDim.x;
        mode[j] = 0;
        X[j] = 0;
        if (i < head) {
            X[j] = bnear[i];
            mode[j] = 1;
        } else if (i < rows) {
            const int64_t k = i - head;
            X[j] = ilist[k];
            mode[j] = 1;
            if (after && k >= nred) {
                const int64_t b = k - nred;
                mode[j] = ((bmask[b >> 5] >> (b & 31)) & 1u) ? 0 : 2;
            }
        }
    }
    pdl_begin();
    double s2 = 0.0;
    long long mxb = 0;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        if (mode[j] == 0) continue;
        const T v = mode[j] == 1 ? residual_int<D, T>(X[j], u, F, G) : T(0);
        r[pos(X[j], G.lay)] = v;
        s2 = fma((double)v, (double)v, s2);
        mxb = max(mxb, abs_bits((double)v));
    }
    if (part) block_partials(s2, mxb, part, blockIdx.x, true);
}

// r = g - B u on the ghost rows (eq. BCh); norm partials at slot0 + block.
// Ctl: the instance that may run the solve control (it holds the device
// graph call; the other instance does not, so profilers list it)
template <int D, typename T, bool Ctl>
__global__ void __launch_bounds__(kT) k_residual_gh(const uint32_t *__restrict__ gidx,
                                                    const uint16_t *__restrict__ gcode, const T *__restrict__ gw,
                                                    int64_t ng, const T *__restrict__ u, const T *__restrict__ F,
                                                    T *__restrict__ r, G2 G, double *__restrict__ part,
                                                    int64_t slot0, NormTail nt, int early) {
    double s2 = 0.0;
    long long mxb = 0;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = g < ng;
    const int64_t X = on ? gidx[g] : 0;
    const uint16_t code = on ? gcode[g] : 0;
    T w[(D == 3) ? 27 : 9];
    ghost_weights<D, T>(code, gw, ng, on ? g : 0, w);
    // early: the predecessor is the interior-row kernel of the same
    // residual, which neither reads nor writes what the ghost rows touch; u
    // and F were written by grids before it, which are complete once this
    // grid runs (see pdl_begin).  So the ghost rows (and their partials) are
    // computed while the interior rows still run, reading u and F through L2;
    // only the final reduction waits for them.
    if (!early) pdl_begin();
    if (on) {
        const int64_t x = pos(X, G.lay);
        const T v = early ? ldv<true>(F + x) - ghost_Bw<D, T, true>(X, code, w, u, G)
                          : F[x] - ghost_Bw<D, T>(X, code, w, u, G);
        r[x] = v;
        s2 = (double)v * (double)v;
        mxb = abs_bits((double)v);
    }
    if (part) block_partials(s2, mxb, part, slot0 + blockIdx.x, false);
    if (early) pdl_begin();
    if (nt.mode) norm_tail<Ctl>(nt, part);
}

template <typename T>
__global__ void __launch_bounds__(kT) k_extend_ell(const uint32_t *__restrict__ bidx,
                                                   const uint8_t *__restrict__ ecnt,
                                                   const uint32_t *__restrict__ eg, const double *__restrict__ ew,
                                                   int64_t nb, T *a, Lay ly) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = b < nb;
    const uint32_t X = on ? bidx[b] : 0u;
    EllRound<T> R;
    R.c = 0;
    if (on) ell_first<T>(b, ecnt, eg, ew, nb, R);
    pdl_begin();
    if (on) a[pos(X, ly)] = extend_from<T>(b, R, eg, ew, nb, a, ly);
}

// One explicit pseudo-time sweep of dr/dsigma + dr/dn = 0 with upwind
// differences at the largest stable step (used when a band node's expanded
// extension has more than kExtCap terms).
template <typename T>
__global__ void __launch_bounds__(kT) k_extend(const uint32_t *__restrict__ bidx, const int32_t *__restrict__ bref,
                                               const double *__restrict__ bw, int64_t nb, int d, T *a,
                                               const T *__restrict__ in, T *__restrict__ out, int last, Lay ly) {
    pdl_begin();
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    T v = T(0);
    for (int ax = 0; ax < d; ++ax) {
        const int32_t ref = bref[(int64_t)ax * nb + b];
        if (ref == kNoRef) continue;
        T s;
        if (ref < 0) s = a[pos(-(int64_t)ref - 1, ly)];
        else s = in ? in[ref] : T(0);
        v = fma((T)bw[(int64_t)ax * nb + b], s, v);
    }
    if (last) a[pos(bidx[b], ly)] = v;
    else out[b] = v;
}

// F_c from the fine residual on coarse interior nodes (first iblocks) and
// coarse ghosts; uc (the coarse correction) is zeroed on the same nodes.
// fmask_c: the family masks of the coarse rows (interior rows, then ghosts)
template <int D, typename T>
__global__ void __launch_bounds__(kT) k_restrict(const uint32_t *__restrict__ ilist_c, int64_t nint_c,
                                                 unsigned iblocks, const uint32_t *__restrict__ gidx_c,
                                                 int64_t ng_c, const uint32_t *__restrict__ fmask_c,
                                                 const T *__restrict__ rf, T *__restrict__ Fc, T *__restrict__ uc,
                                                 T *__restrict__ Fsc, G2 Gf, G2 Gc, int early) {
    const bool interior = blockIdx.x < iblocks;
    const int64_t i = interior ? (int64_t)blockIdx.x * blockDim.x + threadIdx.x
                               : (int64_t)(blockIdx.x - iblocks) * blockDim.x + threadIdx.x;
    const bool on = i < (interior ? nint_c : ng_c);
    const uint32_t Xc = on ? (interior ? ilist_c[i] : gidx_c[i]) : 0u;
    const uint32_t mask = on ? fmask_c[interior ? i : nint_c + i] : 0u;
    int ic[3];
    coords(Xc, (uint32_t)Gc.n, D, ic);
    // early (the predecessor is the fine level's ghost residual or band
    // extension): coarse interior rows read fine interior residuals only,
    // which complete grids wrote (see pdl_begin), and are restricted before
    // the wait, reading them through L2
    const bool now = early && interior;
    if (!now) pdl_begin();
    if (on) {
        const T fc = now ? restrict_masked<D, T, true>(ic, mask, rf, Gf) : restrict_masked<D, T>(ic, mask, rf, Gf);
        const int64_t xc = pos(Xc, Gc.lay);
        Fc[xc] = fc;
        if (Fsc && interior) Fsc[xc] = scaled_rhs<T>(fc, Gc);
        if (uc) uc[xc] = T(0);
    }
    if (now) pdl_begin();
}

// family masks of every coarse level (one launch); level l of the table
// holds the coarse rows of level l, its fine classes those of level l - 1
struct FamTab {
    const uint32_t *ilist, *gidx;
    int64_t nint, ng;
    const uint8_t *clsf;
    G2 Gf, Gc;
    uint32_t *mask;
    int64_t blk;  // first block
};

template <int D>
__global__ void __launch_bounds__(kT) k_family_masks(const FamTab *__restrict__ tab, int nl) {
    pdl_begin();
    int l = 0;
    for (int q = 1; q < nl; ++q)
        if ((int64_t)blockIdx.x >= tab[q].blk) l = q;
    const FamTab &t = tab[l];
    const int64_t i = ((int64_t)blockIdx.x - t.blk) * blockDim.x + threadIdx.x;
    if (i >= t.nint + t.ng) return;
    const bool interior = i < t.nint;
    const uint32_t Xc = interior ? t.ilist[i] : t.gidx[i - t.nint];
    int ic[3];
    coords(Xc, (uint32_t)t.Gc.n, D, ic);
    t.mask[i] = family_mask<D>(ic, interior, t.clsf, t.Gf);
}

// early (the predecessor is the coarse correction's extension, which writes
// coarse band values only): a fine row none of whose coarse corners is
// inactive (so none is a band node) reads only values of complete grids, and
// is prolonged before the dependency wait; the others after it
template <int D, typename T>
__global__ void __launch_bounds__(kT) k_prolong(const uint32_t *__restrict__ ilist, int64_t nint, unsigned iblocks,
                                                const uint32_t *__restrict__ gidx, int64_t ng,
                                                const T *__restrict__ ec, T *__restrict__ uf, G2 Gf, G2 Gc,
                                                const uint8_t *__restrict__ clsc, int early) {
    const bool inner = blockIdx.x < iblocks;
    const int64_t i = inner ? (int64_t)blockIdx.x * blockDim.x + threadIdx.x
                            : (int64_t)(blockIdx.x - iblocks) * blockDim.x + threadIdx.x;
    const bool on = i < (inner ? nint : ng);
    const uint32_t X = on ? (inner ? ilist[i] : gidx[i]) : 0u;
    int iy[3];
    coords(X, (uint32_t)Gf.n, D, iy);
    bool now = false;
    if (early && on) {
        const int t0 = iy[0] & 1, t1 = iy[1] & 1, t2 = (D == 3) ? (iy[2] & 1) : 0;
        const int64_t C0 = (int64_t)(iy[0] >> 1) + (int64_t)(iy[1] >> 1) * Gc.sy +
                           (D == 3 ? (int64_t)(iy[2] >> 1) * Gc.sz : 0);
        bool band = false;
#pragma unroll
        for (int k = 0; k < ((D == 3) ? 8 : 4); ++k) {
            const int b0 = k & 1, b1 = (k >> 1) & 1, b2 = (k >> 2) & 1;
            if (b0 <= t0 && b1 <= t1 && b2 <= t2) band |= clsc[C0 + b0 + b1 * Gc.sy + b2 * Gc.sz] == CL_INACTIVE;
        }
        now = !band;
    }
    // warp-uniform (no lane does its FP64 work twice): early only when the
    // whole warp can go
    now = __all_sync(0xffffffffu, now || !on) && early;
    if (now && on) {
        // before the wait: corners and u_f through L2 (see pdl_begin)
        const int64_t xf = pos(X, Gf.lay);
        uf[xf] = ldv<true>(uf + xf) + prolong_at<D, T, true>(iy, ec, Gc);
    }
    pdl_begin();
    if (on && !now) uf[pos(X, Gf.lay)] += prolong_at<D, T>(iy, ec, Gc);
}

template <typename T>
__global__ void k_coarse_gather(const uint32_t *__restrict__ act, int64_t nact, const T *__restrict__ r,
                                double *__restrict__ rhs, Lay ly) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t X = j < nact ? act[j] : 0u;
    pdl_begin();
    if (j < nact) rhs[j] = (double)r[pos(X, ly)];
}

// u[act[i]] += (A^-1 rhs)_i, one warp per row (FP64 accumulation)
template <typename T>
__global__ void __launch_bounds__(kT) k_coarse_gemv(const uint32_t *__restrict__ act, int64_t nact,
                                                    const double *__restrict__ Ainv,
                                                    const double *__restrict__ rhs, T *__restrict__ u,
                                                    Lay ly) {
    pdl_begin();
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (i >= nact) return;
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int64_t j = lane; j < nact; j += 32) s = fma(Ainv[i * nact + j], rhs[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) u[pos(act[i], ly)] += (T)s;
}

// reduce the residual kernel's block partials in block order (deterministic)
__global__ void __launch_bounds__(1024) k_norm_final(const double *__restrict__ part, int64_t nparts,
                                                     double *__restrict__ out) {
    pdl_begin();
    __shared__ double sh[4][32];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < nparts; i += blockDim.x) {
        a[0] += part[i * 4 + 0];
        a[1] += part[i * 4 + 1];
        a[2] = fmax(a[2], part[i * 4 + 2]);
        a[3] = fmax(a[3], part[i * 4 + 3]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a[0] += __shfl_down_sync(0xffffffffu, a[0], o);
        a[1] += __shfl_down_sync(0xffffffffu, a[1], o);
        a[2] = fmax(a[2], __shfl_down_sync(0xffffffffu, a[2], o));
        a[3] = fmax(a[3], __shfl_down_sync(0xffffffffu, a[3], o));
    }
    if (lane == 0)
        for (int q = 0; q < 4; ++q) sh[q][warp] = a[q];
    __syncthreads();
    if (warp != 0) return;
    const int nw = blockDim.x >> 5;
    for (int q = 0; q < 4; ++q) a[q] = lane < nw ? sh[q][lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a[0] += __shfl_down_sync(0xffffffffu, a[0], o);
        a[1] += __shfl_down_sync(0xffffffffu, a[1], o);
        a[2] = fmax(a[2], __shfl_down_sync(0xffffffffu, a[2], o));
        a[3] = fmax(a[3], __shfl_down_sync(0xffffffffu, a[3], o));
    }
    if (lane == 0) {
        out[0] = sqrt(a[0]);
        out[1] = sqrt(a[1]);
        out[2] = a[2];
        out[3] = a[3];
    }
}

// Weights of every ghost row, all levels in one launch; FP32 copies for the
// mixed cycle.  Dirichlet (eq. BCh): the tensor-product Lagrange weights of
// the interpolant at Q.  Neumann (Sec. 3.2.2, 4.1): its normal derivative at
// Q, sum_a n_a (-s_a / h) L'(xi_a) prod_{b != a} L(xi_b) (the stencil's local
// coordinate along axis a runs against s_a in steps of h).
struct GwTab {
    const uint16_t *gcode;
    const double *gxi, *gn;
    int64_t ng;
    double h;
    double *gw;
    float *gw32;
    int64_t blk;  // first block of this level
};

__global__ void __launch_bounds__(kT) k_ghost_weights(const GwTab *__restrict__ tab, int nl, int d, int bc) {
    pdl_begin();
    int l = 0;
    for (int i = 1; i < nl; ++i)
        if ((int64_t)blockIdx.x >= tab[i].blk) l = i;
    const GwTab &t = tab[l];
    const int64_t g = ((int64_t)blockIdx.x - t.blk) * blockDim.x + threadIdx.x;
    if (g >= t.ng) return;
    const uint16_t code = t.gcode[g];
    double w[3][3], dw[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, c[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a) {
        if (a < d) {
            const int q = (code >> (3 + 2 * a)) & 3;
            const double xi = t.gxi[(int64_t)a * t.ng + g];
            lagrange<double>(q, xi, w[a]);
            if (q == 2) {
                dw[a][0] = __dsub_rn(xi, 1.5);
                dw[a][1] = __dsub_rn(2.0, __dmul_rn(2.0, xi));
                dw[a][2] = __dsub_rn(xi, 0.5);
            } else if (q == 1) {
                dw[a][0] = -1.0;
                dw[a][1] = 1.0;
            }
            // n_a (-s_a / h): s_a = -1 when bit a of the code is set
            const double sa = ((code >> a) & 1) ? -1.0 : 1.0;
            c[a] = __dmul_rn(t.gn[(int64_t)a * t.ng + g], __ddiv_rn(-sa, t.h));
        } else {
            w[a][0] = 1.0;
            w[a][1] = 0.0;
            w[a][2] = 0.0;
        }
    }
    const int n2 = d == 3 ? 3 : 1;
    for (int o2 = 0; o2 < n2; ++o2)
        for (int o1 = 0; o1 < 3; ++o1)
            for (int o0 = 0; o0 < 3; ++o0) {
                const int o[3] = {o0, o1, o2};
                double v;
                if (bc == BCMG_BC_NEUMANN) {
                    v = 0.0;
                    for (int a = 0; a < d; ++a) {
                        double x = __dmul_rn(c[a], dw[a][o[a]]);
                        for (int b = 0; b < d; ++b)
                            if (b != a) x = __dmul_rn(x, w[b][o[b]]);
                        v = __dadd_rn(v, x);
                    }
                } else {
                    v = __dmul_rn(__dmul_rn(w[2][o2], w[1][o1]), w[0][o0]);
                }
                const int64_t k = (int64_t)((o2 * 3 + o1) * 3 + o0) * t.ng + g;
                t.gw[k] = v;
                if (t.gw32) t.gw32[k] = (float)v;
            }
}

// ------------------------------------------------------------ coarse tail
// Levels tail[0..nl-1] (the last one is the coarsest) of the V-cycle in one
// launch on one thread-block cluster: the same per-node steps as the grid
// kernels, separated by the cluster barrier (release / acquire at cluster
// scope, so global writes of one CTA are seen by the others).  Every list of
// a tail level has at most one entry per thread of the cluster, so thread t
// owns entry t of each list; at the start each CTA stages its threads'
// entries of every level in shared memory, which leaves one dependent global
// access in most phases.  A ghost's relaxed value stays in a register across
// the barrier that separates the Jacobi update from its write-back.  Every
// thread reaches every barrier.
template <typename T>
struct TailLevel {
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
    int ell_rounds;  // ceil(longest expansion / 8)
    const uint8_t *cls;
    const uint32_t *fmask;  // restriction families of this level's rows
    T *u, *F, *r;
    T *Fs;  // scaled right-hand side of the interior rows
    const uint32_t *act;
    int64_t nact;
    const double *Ainv;
    double *crhs;
};

namespace cg = cooperative_groups;

constexpr uint32_t kNone = 0xffffffffu;

// per-level staged entries of one CTA's threads (dynamic shared memory)
struct TailSlots {
    uint32_t *red, *black, *gh, *band, *act, *fmask;  // [level * kTailThreads + thread]
    uint16_t *gcode;
};

__device__ __forceinline__ void tail_sync() { cg::this_cluster().sync(); }

// List entry owned by this thread: whole warps of entries are dealt out
// round-robin over the CTAs (so over the SMs and their FP64 pipes), the
// k-th warp of entries going to CTA k % cs, local warp k / cs.
__device__ __forceinline__ int64_t tail_entry() {
    const int64_t k = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    return k * 32 + (threadIdx.x & 31);
}

// band value of slot b with a fixed number of 8-term rounds: the term loads
// do not wait for the row length, and two rounds go together (their 16
// indices and weights, then their 16 values), so a row of up to 16 terms
// costs two dependent round trips
template <typename T>
__device__ __forceinline__ T extend_fixed(int64_t b, int rounds, const uint8_t *ecnt, const uint32_t *eg,
                                          const double *ew, int64_t nb, const T *a, Lay ly) {
    const int c = ecnt[b];
    T v = T(0);
    for (int r0 = 0; r0 < rounds; r0 += 2) {
        uint32_t e[16];
        double w[16];
        const int nt = (rounds - r0 >= 2) ? 16 : 8;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int64_t q = (int64_t)(r0 * 8 + j) * nb + b;
            e[j] = j < nt ? eg[q] : 0u;
            w[j] = j < nt ? ew[q] : 0.0;
        }
        T x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = (r0 * 8 + j < c) ? a[pos(e[j], ly)] : T(0);
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (r0 * 8 + j < c) v = fma((T)w[j], x[j], v);
    }
    return v;
}

template <int D, typename T>
__device__ void tail_smooth(const TailLevel<T> &A, const TailSlots &S, int l, int nsteps) {
    const int t = threadIdx.x;
    const uint32_t xr = S.red[l * kTailThreads + t], xb = S.black[l * kTailThreads + t];
    // ghosts four lanes each (group g = entry / 4, row = entry % 4)
    const uint32_t xg = S.gh[l * kTailThreads + t];
    const uint16_t code = S.gcode[l * kTailThreads + t];
    const int64_t e = tail_entry(), g = e >> 2;
    const int sub = (int)(e & 3);
    const bool on = xg != kNone;
    // register copies of the level's constants and pointers: the table lives
    // in global memory, and the phases' stores would otherwise force the
    // compiler to read it again for every access
    const G2 G = A.g;
    T *const u = A.u;
    const T *const Fs = A.Fs, *const F = A.F, *const gw = A.gw;
    const double *const gdt = A.gdt;
    const int64_t ng = A.ng;
    // split layout with odd n: red = even index, black = odd
    const bool odd_n = (G.n & 1) && G.lay.s == 1;
    const int64_t xs = pos(xg, G.lay);
    for (int s = 0; s < nsteps; ++s) {
        if (xr != kNone) {
            if (odd_n) smooth_at_par<D, T>(xr, u, Fs, G, 0);
            else smooth_at_s<D, T>(xr, u, Fs, G);
        }
        tail_sync();
        if (xb != kNone) {
            if (odd_n) smooth_at_par<D, T>(xb, u, Fs, G, 1);
            else smooth_at_s<D, T>(xb, u, Fs, G);
        }
        tail_sync();
        const T B = ghost_B4<D, T>(on, sub, xg, code, gw, ng, g, u, G);
        T gv = T(0);
        if (on && sub == 0) gv = fma((T)gdt[g], F[xs] - B, u[xs]);
        tail_sync();
        if (on && sub == 0) u[xs] = gv;
        tail_sync();
    }
}

template <int D, typename T>
__device__ void tail_residual(const TailLevel<T> &A, const TailSlots &S, int l) {
    const int t = threadIdx.x;
    const int64_t i = tail_entry();
    const uint32_t xa = S.act[l * kTailThreads + t];
    const G2 G = A.g;
    const T *const u = A.u, *const F = A.F;
    T *const r = A.r;
    if (xa != kNone && i < A.nint) r[pos(xa, G.lay)] = residual_int<D, T>(xa, u, F, G);
    // ghost rows four lanes each, as in the relaxation
    const uint32_t xg = S.gh[l * kTailThreads + t];
    const int64_t g = i >> 2;
    const int sub = (int)(i & 3);
    const T B = ghost_B4<D, T>(xg != kNone, sub, xg, S.gcode[l * kTailThreads + t], A.gw, A.ng, g, u, G);
    if (xg != kNone && sub == 0) r[pos(xg, G.lay)] = F[pos(xg, G.lay)] - B;
    tail_sync();
}

template <typename T>
__device__ void tail_extend(const TailLevel<T> &A, const TailSlots &S, int l, T *a) {
    const int t = threadIdx.x;
    const uint32_t xb = S.band[l * kTailThreads + t];
    const Lay ly = A.g.lay;
    if (xb != kNone) a[pos(xb, ly)] = extend_fixed<T>(tail_entry(), A.ell_rounds, A.ecnt, A.eg, A.ew, A.nb, a, ly);
    tail_sync();
}

// Schedule of the tail (built on the host): a cycle visit of tail level l
// is DOWN(l) (pre-smoothing, residual, extension, restriction to l + 1 with
// the coarse correction zeroed), gamma visits of level l + 1, then UP(l)
// (extension of the coarse correction, prolongation, post-smoothing); a visit
// of the coarsest level is COARSE (its exact correction).  gamma = 1 gives
// the V-cycle, gamma = 2 the W-cycle (Sec. 2.1).
enum : uint8_t { kOpDown = 0, kOpCoarse = 1, kOpUp = 2 };

template <int D, typename T>
__global__ void __launch_bounds__(kTailThreads, 1) k_tail(const TailLevel<T> *__restrict__ tl, int nl,
                                                          const uint8_t *__restrict__ ops, int nops, int nu1,
                                                          int nu2) {
    extern __shared__ uint32_t tsm[];
    TailSlots S;
    const int n = nl * kTailThreads;
    S.red = tsm;
    S.black = tsm + n;
    S.gh = tsm + 2 * n;
    S.band = tsm + 3 * n;
    S.act = tsm + 4 * n;
    S.fmask = tsm + 5 * n;
    S.gcode = (uint16_t *)(tsm + 6 * n);
    const int t = threadIdx.x;
    const int64_t i = tail_entry();  // the grid is one cluster
    for (int l = 0; l < nl; ++l) {
        const TailLevel<T> &A = tl[l];
        const int k = l * kTailThreads + t;
        S.red[k] = i < A.nred ? A.ilist[i] : kNone;
        S.black[k] = i < A.nint - A.nred ? A.ilist[A.nred + i] : kNone;
        S.gh[k] = (i >> 2) < A.ng ? A.gidx[i >> 2] : kNone;  // four lanes per ghost
        S.gcode[k] = (i >> 2) < A.ng ? A.gcode[i >> 2] : (uint16_t)0;
        S.band[k] = i < A.nb ? A.bidx[i] : kNone;
        S.act[k] = i < A.nint ? A.ilist[i] : (i < A.nint + A.ng ? A.gidx[i - A.nint] : kNone);
        S.fmask[k] = (A.fmask && i < A.nint + A.ng) ? A.fmask[i] : 0u;
    }
    __syncthreads();
    pdl_begin();  // the slots above come from fixed tables only
    // each phase helper appears once in the loop (one copy of its code: the
    // tail runs every phase of a cycle once per launch, so its instruction
    // fetches are mostly cold)
    for (int op = 0; op < nops; ++op) {
        const int kind = ops[2 * op], l = ops[2 * op + 1];
        const TailLevel<T> &A = tl[l];
        if (kind == kOpUp) {  // the coarse correction into level l
            const TailLevel<T> &B = tl[l + 1];
            tail_extend<T>(B, S, l + 1, B.u);
            const uint32_t xa = S.act[l * kTailThreads + t];
            const G2 Ag = A.g, Bg = B.g;
            if (xa != kNone) {
                int iy[3];
                coords(xa, (uint32_t)Ag.n, D, iy);
                A.u[pos(xa, Ag.lay)] += prolong_at<D, T>(iy, B.u, Bg);
            }
            tail_sync();
        }
        if (kind != kOpCoarse) tail_smooth<D, T>(A, S, l, kind == kOpDown ? nu1 : nu2);
        if (kind == kOpUp) continue;
        tail_residual<D, T>(A, S, l);
        if (kind == kOpDown) {  // extension, restriction to level l + 1
            const TailLevel<T> &B = tl[l + 1];
            tail_extend<T>(A, S, l, A.r);
            const uint32_t xc = S.act[(l + 1) * kTailThreads + t];
            const G2 Ag = A.g, Bg = B.g;
            if (xc != kNone) {
                int ic[3];
                coords(xc, (uint32_t)Bg.n, D, ic);
                const T fc = restrict_masked<D, T>(ic, S.fmask[(l + 1) * kTailThreads + t], A.r, Ag);
                const int64_t xs = pos(xc, Bg.lay);
                B.F[xs] = fc;
                if (i < B.nint) B.Fs[xs] = scaled_rhs<T>(fc, Bg);
                B.u[xs] = T(0);
            }
            tail_sync();
        } else {  // coarsest: u += A^-1 r on the active rows
            const Lay ly = A.g.lay;
            if (i < A.nact) A.crhs[i] = (double)A.r[pos(A.act[i], ly)];
            tail_sync();
            const int lane = t & 31;
            const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
            for (int64_t row = i >> 5; row < A.nact; row += nthr >> 5) {  // rows by warp, spread over the SMs
                double sum = 0.0;
                for (int64_t j = lane; j < A.nact; j += 32) sum = fma(A.Ainv[row * A.nact + j], A.crhs[j], sum);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
                if (lane == 0) A.u[pos(A.act[row], ly)] += (T)sum;
            }
            tail_sync();
        }
    }
}

// the schedule of one visit of tail level l (levels 0..nl-1, the last the
// coarsest), appended as (kind, level) pairs
void tail_schedule(int l, int nl, int gamma, std::vector<uint8_t> &ops) {
    if (l == nl - 1) {
        ops.push_back(kOpCoarse);
        ops.push_back((uint8_t)l);
        return;
    }
    ops.push_back(kOpDown);
    ops.push_back((uint8_t)l);
    for (int g = 0; g < gamma; ++g) tail_schedule(l + 1, nl, gamma, ops);
    ops.push_back(kOpUp);
    ops.push_back((uint8_t)l);
}

size_t tail_smem(int nl) { return (size_t)nl * kTailThreads * (6 * sizeof(uint32_t) + sizeof(uint16_t)); }

// The dynamic shared-memory limit is a property of the kernel for the whole
// process, shared by every handle: it is always set to what the deepest
// allowed tail needs (kTailMaxLevels levels, 176 KiB), never to one
// handle's need, so no handle can lower it under another's launches.
constexpr int kTailMaxLevels = 16;

// ------------------------------------------------------------ solve control
// separate launches of the start and the check, for levels without ghosts
__global__ void k_solve_init(SolveState *st, const double *__restrict__ nout, cudaGraphConditionalHandle cond) {
    pdl_begin();
    solve_init_dev(st, nout, cond);
}

__global__ void k_solve_check(SolveState *st, const double *__restrict__ nout, cudaGraphConditionalHandle cond) {
    pdl_begin();
    solve_check_dev(st, nout, cond);
}

// ------------------------------------------------------------ mixed precision
// Start of one refinement step on the finest level: the FP32 right-hand side
// is the FP64 residual rounded to FP32, the FP32 correction starts at zero.
__global__ void __launch_bounds__(kT) k_ir_begin(const uint32_t *__restrict__ ilist, int64_t nint,
                                                 const uint32_t *__restrict__ gidx, int64_t ng,
                                                 const double *__restrict__ r, float *__restrict__ F32,
                                                 float *__restrict__ Fs32, float *__restrict__ e32, G2 G) {
    pdl_begin();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nint + ng) return;
    const int64_t x = pos((i < nint) ? ilist[i] : gidx[i - nint], G.lay);
    const float f = (float)r[x];
    F32[x] = f;
    if (i < nint) Fs32[x] = scaled_rhs<float>(f, G);
    e32[x] = 0.0f;
}

// End of a refinement step: u += e on interior and ghost nodes (FP64).
__global__ void __launch_bounds__(kT) k_ir_update(const uint32_t *__restrict__ ilist, int64_t nint,
                                                  const uint32_t *__restrict__ gidx, int64_t ng,
                                                  const float *__restrict__ e32, double *__restrict__ u,
                                                  Lay ly) {
    pdl_begin();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nint + ng) return;
    const int64_t x = pos((i < nint) ? ilist[i] : gidx[i - nint], ly);
    u[x] += (double)e32[x];
}

// ------------------------------------------------------------ data movement
__global__ void __launch_bounds__(kT) k_copy_active(const uint32_t *__restrict__ ilist, int64_t nint,
                                                    const uint32_t *__restrict__ gidx, int64_t ng,
                                                    const uint32_t *__restrict__ box, int64_t nbox,
                                                    const double *__restrict__ src, double *__restrict__ dst,
                                                    Lay ly, int to_split) {
    pdl_begin();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nint + ng + nbox) return;
    int64_t X;
    if (i < nint) X = ilist[i];
    else if (i < nint + ng) X = gidx[i - nint];
    else X = box[i - nint - ng];
    if (to_split) dst[pos(X, ly)] = src[X];
    else dst[X] = src[pos(X, ly)];
}

__global__ void k_scatter_ghosts(const uint32_t *__restrict__ gidx, int64_t ng, const double *__restrict__ g,
                                 double *__restrict__ F, Lay ly) {
    pdl_begin();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ng) F[pos(gidx[i], ly)] = g[i];
}

__global__ void __launch_bounds__(kT) k_set_interior(const uint32_t *__restrict__ ilist, int64_t nint,
                                                     const double *__restrict__ f, double *__restrict__ F,
                                                     double *__restrict__ Fs, G2 G) {
    pdl_begin();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nint) {
        const int64_t X = ilist[i];
        const double v = f ? f[X] : 0.0;  // the caller's array: dense
        F[pos(X, G.lay)] = v;
        Fs[pos(X, G.lay)] = scaled_rhs<double>(v, G);
    }
}

// level arrays of one precision
template <typename T> struct Arr;
template <> struct Arr<double> {
    static double *u(Level &L) { return L.u; }
    static double *F(Level &L) { return L.F; }
    static double *Fs(Level &L) { return L.Fs; }
    static double *r(Level &L) { return L.r; }
    static double *gtmp(Level &L) { return L.gtmp; }
    static double *bbuf(Level &L) { return L.bbuf; }
    static const double *gw(const Level &L) { return L.gw; }
};
template <> struct Arr<float> {
    static float *u(Level &L) { return L.u32; }
    static float *F(Level &L) { return L.F32; }
    static float *Fs(Level &L) { return L.Fs32; }
    static float *r(Level &L) { return L.r32; }
    static float *gtmp(Level &L) { return L.gtmp32; }
    static float *bbuf(Level &L) { return L.bbuf32; }
    static const float *gw(const Level &L) { return L.gw32; }
};

template <typename T>
void run_tail(Handle &H);

template <typename T>
void vcycle_t(Handle &H, int l, T *u) {
    Level &A = H.L[l];
    if (l == (int)H.L.size() - 1) {
        coarsest_correct<T>(H, A, u, Arr<T>::F(A));
        return;
    }
    if (l > 0 && l == H.tail_start) {
        run_tail<T>(H);
        return;
    }
    Level &B = H.L[l + 1];
    smooth<T>(H, A, u, Arr<T>::F(A), H.o.nu1, Arr<T>::Fs(A));
    residual<T>(H, A, u, Arr<T>::F(A), Arr<T>::r(A), H.o.ordering == BCMG_ORDER_RB && H.o.nu1 > 0);
    extend<T>(H, A, Arr<T>::r(A));
    restrict_to<T>(H, A, B, Arr<T>::r(A), Arr<T>::F(B), Arr<T>::u(B), true, Arr<T>::Fs(B));
    // two-grid correction scheme (Sec. 2.1): the level-1 problem solved by
    // tg_inner V-cycles from zero (with more than two levels; else the
    // coarsest solve below is already exact); otherwise gamma visits
    const bool tg = H.o.cycle == BCMG_CYCLE_TG && l == 0 && H.L.size() > 2;
    const int gamma = tg ? H.o.tg_inner : H.o.cycle == BCMG_CYCLE_W ? 2 : 1;
    for (int g = 0; g < gamma; ++g) vcycle_t<T>(H, l + 1, Arr<T>::u(B));
    extend<T>(H, B, Arr<T>::u(B));
    prolong<T>(H, A, B, Arr<T>::u(B), u, true);
    smooth<T>(H, A, u, Arr<T>::F(A), H.o.nu2, Arr<T>::Fs(A));
}

template <typename T>
TailLevel<T> tail_level(Level &L) {
    TailLevel<T> t;
    t.g = g2_of(L);
    t.ilist = L.ilist;
    t.nred = L.nred;
    t.nint = L.nint;
    t.gidx = L.gidx;
    t.gcode = L.gcode;
    t.gw = Arr<T>::gw(L);
    t.gdt = L.gdt;
    t.ng = L.ng;
    t.bidx = L.bidx;
    t.ecnt = L.ecnt;
    t.eg = L.eg;
    t.ew = L.ew;
    t.nb = L.nb;
    t.ell_rounds = (L.ell_max + 7) / 8;
    t.cls = L.cls;
    t.fmask = L.fmask;
    t.u = Arr<T>::u(L);
    t.F = Arr<T>::F(L);
    t.Fs = Arr<T>::Fs(L);
    t.r = Arr<T>::r(L);
    t.act = L.act;
    t.nact = L.nact;
    t.Ainv = L.Ainv;
    t.crhs = L.crhs;
    return t;
}

template <typename T>
using TailKernel = void (*)(const TailLevel<T> *, int, const uint8_t *, int, int, int);

template <typename T>
TailKernel<T> tail_kernel(int d) {
    return d == 3 ? k_tail<3, T> : k_tail<2, T>;
}

cudaLaunchConfig_t tail_config(Handle &H, int csize, int nl, cudaLaunchAttribute *at, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)csize, 1, 1);
    cfg.blockDim = dim3(kTailThreads, 1, 1);
    cfg.dynamicSmemBytes = tail_smem(nl);
    cfg.stream = H.st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 2 : 1;
    return cfg;
}

// largest cluster (16, else 8) of kTailThreads-thread CTAs with the shared
// memory of the deepest allowed tail that the device can place; 0 if none.
// Queried once per device, dimension and precision (the answer does not
// depend on the handle).
template <typename T>
int tail_cluster_size_query(Handle &H) {
    TailKernel<T> k = tail_kernel<T>(H.d);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tail_smem(kTailMaxLevels)) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    for (int cs : {16, 8}) {
        if (cs > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        cudaLaunchAttribute at[2];
        cudaLaunchConfig_t cfg = tail_config(H, cs, kTailMaxLevels, at, false);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n >= 1) return cs;
        (void)cudaGetLastError();
    }
    return 0;
}

std::mutex g_tail_mu;
std::map<std::tuple<int, int, int>, int> g_tail_cs;

template <typename T>
int tail_cluster_size(Handle &H, int nl) {
    if (nl > kTailMaxLevels) return 0;
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    const auto key = std::make_tuple(dev, H.d, (int)sizeof(T));
    std::lock_guard<std::mutex> lk(g_tail_mu);
    auto it = g_tail_cs.find(key);
    if (it != g_tail_cs.end()) return it->second;
    const int cs = tail_cluster_size_query<T>(H);
    g_tail_cs[key] = cs;
    return cs;
}

template <typename T>
void run_tail(Handle &H) {
    const int nl = (int)H.L.size() - H.tail_start;
    const TailLevel<T> *tab = (const TailLevel<T> *)(sizeof(T) == 8 ? H.tail64 : H.tail32);
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = tail_config(H, H.tail_cluster, nl, at, true);
    check_cuda(cudaLaunchKernelEx(&cfg, tail_kernel<T>(H.d), tab, nl, (const uint8_t *)H.tail_ops, H.tail_nops,
                                  H.o.nu1, H.o.nu2),
               "k_tail");
    count_launch(H);
}

}  // namespace

// ------------------------------------------------------------ host wrappers

// one red (c = 0) or black (c = 1) interior sweep of level L
template <typename T>
static void sweep_colour(Handle &H, Level &L, T *u, const T *F, const T *Fs, int c) {
    const G2 G = g2_of(L);
    const uint32_t *list = L.ilist + (c ? L.nred : 0);
    const int64_t n = c ? L.nint - L.nred : L.nred;
    const int bs = bs_for(H, n);
    // red (c = 0) = even index, black = odd, when n is odd
    const int par = ((L.n & 1) && L.lay.s == 1) ? c : -1;
    if (sizeof(T) == 4 && Fs && par >= 0 && n >= kMultiMin * (int64_t)H.nsm) {
        // FP32 sweep of a large level: a persistent grid (the SMs' resident
        // blocks), two entries per thread and chunk
        constexpr int NPT = 2;
        auto k = L.d == 3 ? k_smooth_pers<3, T, NPT> : k_smooth_pers<2, T, NPT>;
        if (H.pers_blocks == 0) {
            int b = 0;
            check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kT, 0), "occupancy");
            H.pers_blocks = std::max(1, b) * H.nsm;
        }
        launch(H, "k_smooth", k, std::min((unsigned)H.pers_blocks, nblk(n, kT * NPT)), kT, list, n, u, Fs, G, par);
    } else if (L.d == 3) {
        launch(H, "k_smooth", k_smooth<3, T>, nblk(n, bs), bs, list, n, u, F, Fs, G, par);
    } else {
        launch(H, "k_smooth", k_smooth<2, T>, nblk(n, bs), bs, list, n, u, F, Fs, G, par);
    }
}

// nsweeps alternating red / black sweeps of the finest level on the handle's
// working arrays (of its working precision), back to back between two
// events; returns their summed device time (ms).  A measurement of the
// sweep as it runs inside a cycle, where each sweep's start overlaps its
// predecessor's end; it changes only the working copy.
double time_sweeps(Handle &H, int nsweeps) {
    Level &L = H.L[0];
    cudaEvent_t e0, e1;
    check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
    check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
    check_cuda(cudaEventRecord(e0, H.st), "event");
    for (int k = 0; k < nsweeps; ++k) {
        if (H.o.precision == BCMG_PREC_MIXED) sweep_colour<float>(H, L, L.u32, L.F32, L.Fs32, k & 1);
        else sweep_colour<double>(H, L, H.u0, L.F, L.Fs, k & 1);
    }
    check_cuda(cudaEventRecord(e1, H.st), "event");
    check_cuda(cudaEventSynchronize(e1), "event sync");
    float ms = 0.0f;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "event time");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (double)ms;
}

// The sweeps of time_sweeps with u and Fs stored as bfloat16 (temporary
// copies of the working arrays; arithmetic in FP32): a measurement of the
// dominant kernel with 16-bit storage.  The level must be parity-split with
// odd n (the grid levels of an even N).
double time_sweeps_bf16(Handle &H, int nsweeps) {
    Level &L = H.L[0];
    if (!((L.n & 1) && L.lay.s == 1)) throw Error{BCMG_EINVAL, "the finest level is not parity-split with odd n"};
    const int64_t len = split_len(L.nn);
    __nv_bfloat16 *u16 = nullptr, *fs16 = nullptr;
    check_cuda(cudaMallocAsync(&u16, sizeof(__nv_bfloat16) * (size_t)len, H.st), "bf16 copy");
    check_cuda(cudaMallocAsync(&fs16, sizeof(__nv_bfloat16) * (size_t)len, H.st), "bf16 copy");
    const bool mixed = H.o.precision == BCMG_PREC_MIXED;
    if (mixed) {
        launch(H, "k_to_bf16", k_to_bf16<float>, nblk(len, kT), kT, (const float *)L.u32, u16, len);
        launch(H, "k_to_bf16", k_to_bf16<float>, nblk(len, kT), kT, (const float *)L.Fs32, fs16, len);
    } else {
        launch(H, "k_to_bf16", k_to_bf16<double>, nblk(len, kT), kT, (const double *)H.u0, u16, len);
        launch(H, "k_to_bf16", k_to_bf16<double>, nblk(len, kT), kT, (const double *)L.Fs, fs16, len);
    }
    constexpr int NPT = 2;
    auto k = L.d == 3 ? k_smooth_pers_bf16<3, NPT> : k_smooth_pers_bf16<2, NPT>;
    int b = 0;
    check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kT, 0), "occupancy");
    const unsigned resident = (unsigned)(std::max(1, b) * H.nsm);
    const G2 G = g2_of(L);
    cudaEvent_t e0, e1;
    check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
    check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
    check_cuda(cudaEventRecord(e0, H.st), "event");
    for (int s = 0; s < nsweeps; ++s) {
        const int c = s & 1;
        const int64_t n = c ? L.nint - L.nred : L.nred;
        launch(H, "k_smooth", k, std::min(resident, nblk(n, kT * NPT)), kT, (const uint32_t *)(L.ilist + (c ? L.nred : 0)),
               n, u16, (const __nv_bfloat16 *)fs16, G, c);
    }
    check_cuda(cudaEventRecord(e1, H.st), "event");
    check_cuda(cudaEventSynchronize(e1), "event sync");
    float ms = 0.0f;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "event time");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(u16, H.st);
    cudaFreeAsync(fs16, H.st);
    return (double)ms;
}

template <typename T>
void smooth(Handle &H, Level &L, T *u, const T *F, int nsteps, const T *Fs) {
    const G2 G = g2_of(L);
    T *tmp = Arr<T>::gtmp(L);
    const T *gw = Arr<T>::gw(L);
    // the timed sweeps are the finest-level ones of the solve's working precision
    const bool prof = (sizeof(T) == 8) == (H.o.precision == BCMG_PREC_FP64);
    const int bg = bs_for(H, L.ng);
    for (int s = 0; s < nsteps; ++s) {
        if (H.o.ordering == BCMG_ORDER_LEX) {
            // GS-LEX (eq. GSLEX_2D): hyperplanes in increasing p; each node
            // sees new values below it and old values above, as in the
            // lexicographic loop
            for (size_t q = 0; q + 1 < L.hoff.size(); ++q) {
                const int64_t n = L.hoff[q + 1] - L.hoff[q];
                if (n == 0) continue;
                const int bs = bs_for(H, n);
                const uint32_t *list = L.hlist + L.hoff[q];
                // hyperplane p = i + j (+ k) = q: one index parity when n is odd
                const int par = ((L.n & 1) && L.lay.s == 1) ? (int)(q & 1) : -1;
                if (L.d == 3) launch(H, "k_smooth", k_smooth<3, T>, nblk(n, bs), bs, list, n, u, F, Fs, G, par);
                else launch(H, "k_smooth", k_smooth<2, T>, nblk(n, bs), bs, list, n, u, F, Fs, G, par);
            }
        }
        for (int c = 0; c < 2 && H.o.ordering == BCMG_ORDER_RB; ++c) {
            if (prof) profile_mark(H, L);
            sweep_colour<T>(H, L, u, F, Fs, c);
            if (prof) profile_mark(H, L);
        }
        if (L.d == 3)
            launch(H, "k_ghost_relax", k_ghost_relax<3, T>, nblk(L.ng, bg), bg, (const uint32_t *)L.gidx,
                   (const uint16_t *)L.gcode, gw, (const double *)L.gdt, L.ng, (const T *)u, F, tmp, G);
        else
            launch(H, "k_ghost_relax", k_ghost_relax<2, T>, nblk(L.ng, bg), bg, (const uint32_t *)L.gidx,
                   (const uint16_t *)L.gcode, gw, (const double *)L.gdt, L.ng, (const T *)u, F, tmp, G);
        launch(H, "k_ghost_scatter", k_ghost_scatter<T>, nblk(L.ng, bg), bg, (const uint32_t *)L.gidx, L.ng,
               (const T *)tmp, u, L.lay);
    }
}

// interior rows, then ghost rows (separate kernels: the ghost stencil's
// registers would otherwise limit the occupancy of the interior rows);
// returns the number of norm partials written
template <typename T>
static int64_t residual_impl(Handle &H, Level &L, const T *u, const T *F, T *r, double *part,
                             NormTail nt = NormTail{}, bool after_rb = false) {
    const G2 G = g2_of(L);
    const int64_t rows = after_rb ? L.nint + L.nbn : L.nint;
    // with norm partials, kNormRows interior rows per thread; with the norm
    // tail, full-size ghost blocks (the last one reduces every partial)
    constexpr int kNormRows = 4;
    const int npt = part ? kNormRows : 1;
    const int bi = bs_for(H, (rows + npt - 1) / npt), bg = nt.mode ? kT : bs_for(H, L.ng);
    const int64_t ni = nblk(rows, bi * npt);
    const T *gw = Arr<T>::gw(L);
    nt.nparts = ni + nblk(L.ng, bg);
    if (L.d == 3) {
        launch(H, "k_residual_int", part ? k_residual_int<3, T, kNormRows> : k_residual_int<3, T, 1>, (unsigned)ni,
               bi, (const uint32_t *)L.ilist, L.nint, L.nred, (const uint32_t *)L.bmask,
               (const uint32_t *)L.bnear, L.nbn, (int)after_rb, u, F, r, G, part);
        if (L.ng == 0) return ni;
        launch(H, "k_residual_gh", nt.mode > 1 ? k_residual_gh<3, T, true> : k_residual_gh<3, T, false>,
               nblk(L.ng, bg), bg, (const uint32_t *)L.gidx, (const uint16_t *)L.gcode, gw, L.ng, u, F, r, G, part,
               ni, nt, (int)(ni > 0));
    } else {
        launch(H, "k_residual_int", part ? k_residual_int<2, T, kNormRows> : k_residual_int<2, T, 1>, (unsigned)ni,
               bi, (const uint32_t *)L.ilist, L.nint, L.nred, (const uint32_t *)L.bmask,
               (const uint32_t *)L.bnear, L.nbn, (int)after_rb, u, F, r, G, part);
        if (L.ng == 0) return ni;
        launch(H, "k_residual_gh", nt.mode > 1 ? k_residual_gh<2, T, true> : k_residual_gh<2, T, false>,
               nblk(L.ng, bg), bg, (const uint32_t *)L.gidx, (const uint16_t *)L.gcode, gw, L.ng, u, F, r, G, part,
               ni, nt, (int)(ni > 0));
    }
    return ni + nblk(L.ng, bg);
}

template <typename T>
void residual(Handle &H, Level &L, const T *u, const T *F, T *r, bool after_rb) {
    residual_impl<T>(H, L, u, F, r, nullptr, NormTail{}, after_rb);
}

template <typename T>
void extend(Handle &H, Level &L, T *a) {
    if (L.nb == 0) return;
    const int bs = bs_for(H, L.nb);
    if (L.ecnt) {
        launch(H, "k_extend_ell", k_extend_ell<T>, nblk(L.nb, bs), bs, (const uint32_t *)L.bidx,
               (const uint8_t *)L.ecnt, (const uint32_t *)L.eg, (const double *)L.ew, L.nb, a, L.lay);
        return;
    }
    const int K = std::max(H.o.ext_sweeps, 1);
    T *b0 = Arr<T>::bbuf(L), *b1 = Arr<T>::bbuf(L) + L.nb;
    const T *in = nullptr;
    for (int k = 0; k < K; ++k) {
        const int last = (k == K - 1);
        T *out = (k % 2 == 0) ? b0 : b1;
        launch(H, "k_extend", k_extend<T>, nblk(L.nb, bs), bs, (const uint32_t *)L.bidx, (const int32_t *)L.bref,
               (const double *)L.bw, L.nb, L.d, a, in, out, last, L.lay);
        in = out;
    }
}

template <typename T>
void restrict_to(Handle &H, Level &Lf, Level &Lc, const T *rf, T *Fc, T *uc_zero, bool early_ok, T *Fsc) {
    const G2 Gf = g2_of(Lf), Gc = g2_of(Lc);
    const int bs = bs_for(H, Lc.nint + Lc.ng);
    const unsigned ib = nblk(Lc.nint, bs);
    const unsigned grid = ib + nblk(Lc.ng, bs);
    // in the cycle the fine residual's interior rows are at least two
    // launches back when the level has ghost rows or a band
    const int early = (int)(early_ok && (Lf.ng > 0 || Lf.nb > 0));
    if (Lf.d == 3)
        launch(H, "k_restrict", k_restrict<3, T>, grid, bs, (const uint32_t *)Lc.ilist, Lc.nint, ib,
               (const uint32_t *)Lc.gidx, Lc.ng, (const uint32_t *)Lc.fmask, rf, Fc, uc_zero, Fsc, Gf, Gc, early);
    else
        launch(H, "k_restrict", k_restrict<2, T>, grid, bs, (const uint32_t *)Lc.ilist, Lc.nint, ib,
               (const uint32_t *)Lc.gidx, Lc.ng, (const uint32_t *)Lc.fmask, rf, Fc, uc_zero, Fsc, Gf, Gc, early);
}

template <typename T>
void prolong(Handle &H, Level &Lf, Level &Lc, const T *ec, T *uf, bool early_ok) {
    const G2 Gf = g2_of(Lf), Gc = g2_of(Lc);
    const int bs = bs_for(H, Lf.nint + Lf.ng);
    const unsigned ib = nblk(Lf.nint, bs);
    const unsigned grid = ib + nblk(Lf.ng, bs);
    // the cycle extends the coarse correction right before (when the
    // coarse level has a band); a caller's own prolongation has no
    // predecessor on the library stream
    const int early = (int)(early_ok && Lc.nb > 0);
    if (Lf.d == 3)
        launch(H, "k_prolong", k_prolong<3, T>, grid, bs, (const uint32_t *)Lf.ilist, Lf.nint, ib,
               (const uint32_t *)Lf.gidx, Lf.ng, ec, uf, Gf, Gc, (const uint8_t *)Lc.cls, early);
    else
        launch(H, "k_prolong", k_prolong<2, T>, grid, bs, (const uint32_t *)Lf.ilist, Lf.nint, ib,
               (const uint32_t *)Lf.gidx, Lf.ng, ec, uf, Gf, Gc, (const uint8_t *)Lc.cls, early);
}

template <typename T>
void coarsest_correct(Handle &H, Level &L, T *u, const T *F) {
    residual<T>(H, L, u, F, Arr<T>::r(L));
    launch(H, "k_coarse_gather", k_coarse_gather<T>, nblk(L.nact, 64), 64, (const uint32_t *)L.act, L.nact,
           (const T *)Arr<T>::r(L), L.crhs, L.lay);
    launch(H, "k_coarse_gemv", k_coarse_gemv<T>, nblk(L.nact, 2), 64, (const uint32_t *)L.act, L.nact,
           (const double *)L.Ainv, (const double *)L.crhs, u, L.lay);
}

// residual of the finest level and its four norms, optionally followed by
// the solve's start (ctl 1) or per-cycle check (ctl 2).  With ghosts, the
// last block of the ghost residual kernel reduces the block partials and
// runs the control; without, a single-block reduction and a separate
// control launch follow.
void residual_norms(Handle &H, const double *u, double *out4, int ctl, unsigned long long cond, bool after_rb) {
    Level &L = H.L[0];
    if (L.ng > 0) {
        NormTail nt{};
        nt.mode = 1 + ctl;
        nt.counter = H.ncount;
        nt.nout = out4;
        nt.st = H.sdev;
        nt.cond = (cudaGraphConditionalHandle)cond;
        residual_impl<double>(H, L, u, L.F, L.r, H.npart, nt, after_rb);
        return;
    }
    const int64_t parts = residual_impl<double>(H, L, u, L.F, L.r, H.npart, NormTail{}, after_rb);
    launch(H, "k_norm_final", k_norm_final, 1u, 1024u, (const double *)H.npart, parts, out4);
    if (ctl == 1) solve_init_enqueue(H, cond);
    else if (ctl == 2) solve_check_enqueue(H, cond);
}

// an upper bound of the block partials residual_norms writes (64-thread blocks)
int64_t norm_parts(const Level &L) { return (int64_t)nblk(L.nint + L.nbn, 64) + nblk(L.ng, 64); }

// V(nu1, nu2) cycle from level l down (Sec. 2.1 with gamma = 1); u is the
// level's unknown (finest: the working copy, coarse: the correction).
void vcycle_enqueue(Handle &H, int l, double *u) { vcycle_t<double>(H, l, u); }

void mixed_step_enqueue(Handle &H, double *u) {
    Level &L = H.L[0];
    const unsigned grid = nblk(L.nint + L.ng, kT);
    launch(H, "k_ir_begin", k_ir_begin, grid, kT, (const uint32_t *)L.ilist, L.nint, (const uint32_t *)L.gidx, L.ng,
           (const double *)L.r, L.F32, L.Fs32, L.u32, g2_of(L));
    vcycle_t<float>(H, 0, L.u32);
    launch(H, "k_ir_update", k_ir_update, grid, kT, (const uint32_t *)L.ilist, L.nint, (const uint32_t *)L.gidx,
           L.ng, (const float *)L.u32, u, L.lay);
}

// Cycle tables made once after the hierarchy: the ghost interpolation
// weights of every level (one launch), then the levels of the cluster tail
// and their tables.  The tail holds the coarse levels whose interior +
// ghost + band nodes fit kTailNodes and whose extension is expanded (ELL),
// down to a coarsest level of at most kTailCoarse unknowns; it needs a level
// above the coarsest and never starts at level 0.
void setup_cycle(Handle &H) {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    check_cuda(cudaDeviceGetAttribute(&H.nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int L = (int)H.L.size();
    const bool mixed = H.o.precision == BCMG_PREC_MIXED;
    const int nterm = H.d == 3 ? 27 : 9;
    std::vector<GwTab> gt(L);
    int64_t blocks = 0;
    // the weight tables of every level (zero outside each ghost's stencil
    // degrees): slices of one zero-filled block
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t wbytes = 0;
    for (int l = 0; l < L; ++l) {
        const size_t n1 = (size_t)std::max<int64_t>(H.L[l].ng, 1) * nterm;
        wbytes += al(sizeof(double) * n1) + (mixed ? al(sizeof(float) * n1) : 0);
    }
    char *wnext = (char *)dalloc(H, wbytes);
    for (int l = 0; l < L; ++l) {
        Level &A = H.L[l];
        const size_t n1 = (size_t)std::max<int64_t>(A.ng, 1) * nterm;
        A.gw = (double *)wnext;
        wnext += al(sizeof(double) * n1);
        if (mixed) {
            A.gw32 = (float *)wnext;
            wnext += al(sizeof(float) * n1);
        }
        gt[l] = GwTab{A.gcode, A.gxi, A.gn, A.ng, A.h, A.gw, A.gw32, blocks};
        blocks += nblk(A.ng, kT);
    }
    if (blocks > 0) {
        GwTab *gt_d = (GwTab *)dalloc(H, sizeof(GwTab) * L, true);
        check_cuda(cudaMemcpyAsync(gt_d, gt.data(), sizeof(GwTab) * L, cudaMemcpyHostToDevice, H.st), "gw table");
        launch(H, "k_ghost_weights", k_ghost_weights, (unsigned)blocks, kT, (const GwTab *)gt_d, L, H.d, H.o.bc);
    }
    // restriction families of the coarse rows, every coarse level in one launch
    if (L > 1) {
        std::vector<FamTab> ft(L - 1);
        int64_t fblocks = 0;
        for (int l = 1; l < L; ++l) {
            Level &C = H.L[l], &F = H.L[l - 1];
            C.fmask = (uint32_t *)dalloc(H, sizeof(uint32_t) * (size_t)std::max<int64_t>(C.nint + C.ng, 1), false,
                                         false);
            ft[l - 1] = FamTab{C.ilist, C.gidx, C.nint, C.ng, F.cls, g2_of(F), g2_of(C), C.fmask, fblocks};
            fblocks += nblk(C.nint + C.ng, kT);
        }
        if (fblocks > 0) {
            FamTab *ft_d = (FamTab *)dalloc(H, sizeof(FamTab) * (L - 1), true);
            check_cuda(cudaMemcpyAsync(ft_d, ft.data(), sizeof(FamTab) * (L - 1), cudaMemcpyHostToDevice, H.st),
                       "family table");
            if (H.d == 3)
                launch(H, "k_family_masks", k_family_masks<3>, (unsigned)fblocks, kT, (const FamTab *)ft_d, L - 1);
            else
                launch(H, "k_family_masks", k_family_masks<2>, (unsigned)fblocks, kT, (const FamTab *)ft_d, L - 1);
        }
    }

    // a level fits the tail if each of its lists has at most one entry per
    // thread of the cluster (four threads per ghost; at most kTailNodes) and
    // its extension is expanded; the coarsest level also needs at most
    // kTailCoarse unknowns
    H.tail_start = -1;
    if (H.o.ordering != BCMG_ORDER_RB) return;  // the tail runs red-black sweeps
    auto fits = [&](const Level &A, int64_t lim) {
        return A.nint + A.ng <= lim && 4 * A.ng <= lim && A.nb <= lim && (A.nb == 0 || A.ecnt != nullptr);
    };
    auto first_level = [&](int64_t lim) {
        int lt = L - 1;
        while (lt - 1 >= 1 && fits(H.L[lt - 1], lim)) --lt;
        return lt;
    };
    const Level &C = H.L[L - 1];
    int lt = first_level(kTailNodes);
    if (lt >= L - 1 || !fits(C, kTailNodes) || C.nact > kTailCoarse) return;
    const int cs = tail_cluster_size<double>(H, L - lt);
    if (cs == 0 || (mixed && tail_cluster_size<float>(H, L - lt) < cs)) return;
    const int64_t lim = std::min<int64_t>(kTailNodes, (int64_t)cs * kTailThreads);
    lt = std::max(lt, first_level(lim));
    if (lt >= L - 1 || !fits(C, lim) || C.nact > lim) return;
    H.tail_cluster = cs;
    H.tail_start = lt;
    const int nl = L - lt;
    // the tail's levels keep the dense layout (nothing has been written to
    // their value arrays yet; zeros read the same in either layout)
    for (int l = lt; l < L; ++l) H.L[l].lay = Lay{0u, 0u, 0u};
    std::vector<uint8_t> ops;
    tail_schedule(0, nl, H.o.cycle == BCMG_CYCLE_W ? 2 : 1, ops);
    H.tail_nops = (int)(ops.size() / 2);
    H.tail_ops = dalloc(H, ops.size());
    check_cuda(cudaMemcpyAsync(H.tail_ops, ops.data(), ops.size(), cudaMemcpyHostToDevice, H.st), "tail schedule");
    std::vector<TailLevel<double>> t64;
    for (int l = lt; l < L; ++l) t64.push_back(tail_level<double>(H.L[l]));
    H.tail64 = dalloc(H, sizeof(TailLevel<double>) * nl);
    check_cuda(cudaMemcpyAsync(H.tail64, t64.data(), sizeof(TailLevel<double>) * nl, cudaMemcpyHostToDevice, H.st),
               "tail table");
    if (mixed) {
        std::vector<TailLevel<float>> t32;
        for (int l = lt; l < L; ++l) t32.push_back(tail_level<float>(H.L[l]));
        H.tail32 = dalloc(H, sizeof(TailLevel<float>) * nl);
        check_cuda(cudaMemcpyAsync(H.tail32, t32.data(), sizeof(TailLevel<float>) * nl, cudaMemcpyHostToDevice,
                                   H.st),
                   "tail table");
    }
}

void solve_init_enqueue(Handle &H, unsigned long long cond) {
    launch(H, "k_solve_init", k_solve_init, 1u, 1u, H.sdev, (const double *)H.nout, (cudaGraphConditionalHandle)cond);
}

void solve_check_enqueue(Handle &H, unsigned long long cond) {
    launch(H, "k_solve_check", k_solve_check, 1u, 1u, H.sdev, (const double *)H.nout,
           (cudaGraphConditionalHandle)cond);
}

void copy_active(Handle &H, const double *src, double *dst, bool in) {
    Level &L = H.L[0];
    const bool with_boxdir = in;
    const int64_t nbox = with_boxdir ? L.nbox : 0;
    launch(H, "k_copy_active", k_copy_active, nblk(L.nint + L.ng + nbox, kT), kT, (const uint32_t *)L.ilist, L.nint,
           (const uint32_t *)L.gidx, L.ng, (const uint32_t *)L.boxidx, nbox, src, dst, L.lay, (int)with_boxdir);
}

namespace {
__global__ void __launch_bounds__(kT) k_permute(const double *__restrict__ src, double *__restrict__ dst, int64_t nn,
                                                Lay ly, int to_split) {
    pdl_begin();
    const int64_t X = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= nn) return;
    if (to_split) dst[pos(X, ly)] = src[X];
    else dst[X] = src[pos(X, ly)];
}
}  // namespace

void dense_to_split(Handle &H, const Level &L, const double *dense, double *split) {
    launch(H, "k_permute", k_permute, nblk(L.nn, kT), kT, dense, split, L.nn, L.lay, 1);
}

void split_to_dense(Handle &H, const Level &L, const double *split, double *dense) {
    launch(H, "k_permute", k_permute, nblk(L.nn, kT), kT, split, dense, L.nn, L.lay, 0);
}

void scatter_ghost_values(Handle &H, Level &L, const double *g, double *F) {
    launch(H, "k_scatter_ghosts", k_scatter_ghosts, nblk(L.ng, kT), kT, (const uint32_t *)L.gidx, L.ng, g, F, L.lay);
}

void set_interior_rhs(Handle &H, Level &L, const double *f, double *F) {
    launch(H, "k_set_interior", k_set_interior, nblk(L.nint, kT), kT, (const uint32_t *)L.ilist, L.nint, f, F,
           L.Fs, g2_of(L));
}

namespace {
template <typename T>
__global__ void k_div_wsum_test(const double *__restrict__ a, int64_t n, double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)div_wsum<T>((T)a[i], (int)(1 + i % 64));
}
}  // namespace

int selftest_div_wsum(int fp32, const double *a_host, int64_t n, double *out_host, std::string *msg) {
    if (!a_host || !out_host || n < 1 || n > (1 << 24)) {
        *msg = "null pointer or n outside [1, 2^24]";
        return BCMG_EINVAL;
    }
    double *buf = nullptr;
    const size_t bytes = (size_t)n * sizeof(double);
    if (cudaMalloc(&buf, 2 * bytes) != cudaSuccess) {
        *msg = "cudaMalloc failed";
        return BCMG_ENOMEM;
    }
    int rc = BCMG_OK;
    cudaError_t e = cudaMemcpy(buf, a_host, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (fp32) k_div_wsum_test<float><<<nblk(n, 256), 256>>>(buf, n, buf + n);
        else k_div_wsum_test<double><<<nblk(n, 256), 256>>>(buf, n, buf + n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out_host, buf + n, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        *msg = std::string("selftest_div_wsum: ") + cudaGetErrorString(e);
        rc = BCMG_ECUDA;
    }
    cudaFree(buf);
    add_launches(1);
    return rc;
}

template void smooth<double>(Handle &, Level &, double *, const double *, int, const double *);
template void residual<double>(Handle &, Level &, const double *, const double *, double *, bool);
template void extend<double>(Handle &, Level &, double *);
template void restrict_to<double>(Handle &, Level &, Level &, const double *, double *, double *, bool, double *);
template void prolong<double>(Handle &, Level &, Level &, const double *, double *, bool);
template void coarsest_correct<double>(Handle &, Level &, double *, const double *);
template void smooth<float>(Handle &, Level &, float *, const float *, int, const float *);
template void residual<float>(Handle &, Level &, const float *, const float *, float *, bool);
template void extend<float>(Handle &, Level &, float *);
template void restrict_to<float>(Handle &, Level &, Level &, const float *, float *, float *, bool, float *);
template void prolong<float>(Handle &, Level &, Level &, const float *, float *, bool);
template void coarsest_correct<float>(Handle &, Level &, float *, const float *);

}  // namespace bcmg

extern "C" int bcmg_selftest_div_wsum(int fp32, const double *a_host, int64_t n, double *out_host) {
    std::string msg;
    int rc = bcmg::selftest_div_wsum(fp32, a_host, n, out_host, &msg);
    return bcmg::report(rc, msg);
}
