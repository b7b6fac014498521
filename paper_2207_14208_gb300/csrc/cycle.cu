// Multigrid cycle kernels of the GB300 BCMG library (arXiv 2207.14208).
//
// Interior work runs over the compacted 64-node windows (one warp per
// window, coalesced x-rows, no class reads); ghost and band work over their
// compacted lists.  All kernels are FP64 and memory- or FP64-ALU bound; none
// is a dense contraction, so no tensor-core path is used.
#include <algorithm>

#include "bcmg_internal.cuh"

namespace bcmg {

namespace {

struct G2 {
    int d, N, n;
    int64_t sy, sz;
    double h2, ih2, inv2d;
};

G2 g2_of(const Level &L) {
    G2 g;
    g.d = L.d;
    g.N = L.N;
    g.n = L.n;
    g.sy = L.st[1];
    g.sz = L.st[2];
    g.h2 = L.h * L.h;
    g.ih2 = 1.0 / g.h2;
    g.inv2d = 1.0 / (2.0 * L.d);
    return g;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
inline unsigned wblk(int64_t nwin) { return (unsigned)((nwin + kWarpsPerBlock - 1) / kWarpsPerBlock); }
constexpr int kT = kWarpsPerBlock * 32;

#define LAUNCH(kern, grid, block, ...)                                   \
    do {                                                                \
        if ((grid) > 0) {                                               \
            kern<<<(grid), (block), 0, H.st>>>(__VA_ARGS__);            \
            check_cuda(cudaGetLastError(), #kern);                      \
            count_launch(H);                                            \
        }                                                               \
    } while (0)

__device__ __forceinline__ void lagrange(int q, double xi, double w[3]) {
    // quadratic / linear / constant Lagrange basis on local nodes 0, 1, 2
    // (eq. coeff: c_0, c_-1, c_-2 at xi = theta)
    if (q == 2) {
        w[0] = (1.0 - xi) * (2.0 - xi) * 0.5;
        w[1] = xi * (2.0 - xi);
        w[2] = xi * (xi - 1.0) * 0.5;
    } else if (q == 1) {
        w[0] = 1.0 - xi;
        w[1] = xi;
        w[2] = 0.0;
    } else {
        w[0] = 1.0;
        w[1] = 0.0;
        w[2] = 0.0;
    }
}

// B u~ at a ghost: the (tri/bi)quadratic interpolant on ST_G at Q (eq. BCh).
// Fully unrolled with compile-time stencil offsets (weights stay in
// registers); nodes beyond an axis' degree are never loaded.
template <int D>
__device__ __forceinline__ double ghost_B(int64_t X, uint16_t code, const double *__restrict__ gxi, int64_t ng,
                                          int64_t g, const double *u, const G2 &G) {
    const int qx = (code >> 3) & 3, qy = (code >> 5) & 3, qz = (D == 3) ? ((code >> 7) & 3) : 0;
    const int64_t ox = (code & 1) ? 1 : -1;
    const int64_t oy = (code & 2) ? G.sy : -G.sy;
    const int64_t oz = (D == 3) ? ((code & 4) ? G.sz : -G.sz) : 0;
    double wx[3], wy[3], wz[3] = {1.0, 0.0, 0.0};
    lagrange(qx, gxi[g], wx);
    lagrange(qy, gxi[ng + g], wy);
    if (D == 3) lagrange(qz, gxi[2 * ng + g], wz);
    double B = 0.0;
#pragma unroll
    for (int o2 = 0; o2 < (D == 3 ? 3 : 1); ++o2) {
        if (o2 > qz) break;
#pragma unroll
        for (int o1 = 0; o1 < 3; ++o1) {
            if (o1 > qy) break;
            const double wyz = wz[o2] * wy[o1];
            const int64_t Y = X + o2 * oz + o1 * oy;
#pragma unroll
            for (int o0 = 0; o0 < 3; ++o0) {
                if (o0 > qx) break;
                B = fma(wyz * wx[o0], u[Y + o0 * ox], B);
            }
        }
    }
    return B;
}

template <int D>
__device__ __forceinline__ double nbr_sum(const double *u, int64_t X, const G2 &G) {
    double s = (u[X - 1] + u[X + 1]) + (u[X - G.sy] + u[X + G.sy]);
    if (D == 3) s += u[X - G.sz] + u[X + G.sz];
    return s;
}

// ------------------------------------------------------------ smoothing
// One colour of red-black Gauss-Seidel on interior nodes (eq. GSLEX_2D in
// red-black order): u_X = (sum of 2d neighbours + h^2 F_X) / (2d).
template <int D>
__global__ void __launch_bounds__(kT) k_smooth(const Win *__restrict__ win, int64_t nwin, double *u,
                                               const double *__restrict__ F, G2 G, int color) {
    int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= nwin) return;
    const int lane = threadIdx.x & 31;
    const Win W = win[w];
    const int par = ((W.jk & 0xffffu) + (W.jk >> 16)) & 1;
    const int t = 2 * lane + ((color ^ par) & 1);
    if (!((W.mask >> t) & 1ull)) return;
    const int64_t X = (int64_t)W.base + t;
    const double s = nbr_sum<D>(u, X, G);
    u[X] = fma(G.h2, F[X], s) * G.inv2d;
}

// Fictitious-time relaxation of all ghosts from the same u (eq. rel with
// eq. DtauOptTheta; the ghost block of P is diag(1/Delta tau)): new values go
// to tmp, then k_ghost_scatter writes them.
template <int D>
__global__ void k_ghost_relax(const uint32_t *__restrict__ gidx, const uint16_t *__restrict__ gcode,
                              const double *__restrict__ gxi, const double *__restrict__ gdt, int64_t ng,
                              const double *u, const double *__restrict__ F, double *__restrict__ tmp, G2 G) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int64_t X = gidx[g];
    const double B = ghost_B<D>(X, gcode[g], gxi, ng, g, u, G);
    tmp[g] = fma(gdt[g], F[X] - B, u[X]);
}

__global__ void k_ghost_scatter(const uint32_t *__restrict__ gidx, int64_t ng, const double *__restrict__ tmp,
                                double *__restrict__ u) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    u[gidx[g]] = tmp[g];
}

// ------------------------------------------------------------ residual
// r = F - A u on interior rows (eq. Laph) and ghost rows (eq. BCh).
template <int D>
__global__ void __launch_bounds__(kT) k_residual(const Win *__restrict__ win, int64_t nwin, unsigned wblocks,
                                                 const uint32_t *__restrict__ gidx,
                                                 const uint16_t *__restrict__ gcode,
                                                 const double *__restrict__ gxi, int64_t ng,
                                                 const double *__restrict__ u, const double *__restrict__ F,
                                                 double *__restrict__ r, G2 G) {
    if (blockIdx.x < wblocks) {
        int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (w >= nwin) return;
        const int lane = threadIdx.x & 31;
        const Win W = win[w];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = lane + 32 * h;
            if (!((W.mask >> t) & 1ull)) continue;
            const int64_t X = (int64_t)W.base + t;
            const double s = nbr_sum<D>(u, X, G);
            r[X] = F[X] - (2.0 * D * u[X] - s) * G.ih2;
        }
        return;
    }
    int64_t g = (int64_t)(blockIdx.x - wblocks) * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int64_t X = gidx[g];
    r[X] = F[X] - ghost_B<D>(X, gcode[g], gxi, ng, g, u, G);
}

// ------------------------------------------------------------ band extension
// One explicit pseudo-time sweep of dr/dsigma + dr/dn = 0 with upwind
// differences at the largest stable step: each band value becomes the
// normalised |n_a|-weighted mean of its upwind ghost / band sources.
__global__ void k_extend(const uint32_t *__restrict__ bidx, const int32_t *__restrict__ bref,
                         const double *__restrict__ bw, int64_t nb, int d, double *a,
                         const double *__restrict__ in, double *__restrict__ out, int last) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double v = 0.0;
    for (int ax = 0; ax < d; ++ax) {
        const int32_t ref = bref[(int64_t)ax * nb + b];
        if (ref == kNoRef) continue;
        double s;
        if (ref < 0) s = a[-(int64_t)ref - 1];
        else s = in ? in[ref] : 0.0;
        v = fma(bw[(int64_t)ax * nb + b], s, v);
    }
    if (last) a[bidx[b]] = v;
    else out[b] = v;
}

// All K sweeps at once: band value = sum over the precomputed (ghost, weight)
// row of the band node (the expansion of the sweeps started from zero).
__global__ void k_extend_csr(const uint32_t *__restrict__ bidx, const int64_t *__restrict__ eoff,
                             const uint32_t *__restrict__ eg, const double *__restrict__ ew, int64_t nb,
                             double *a) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double v = 0.0;
    for (int64_t j = eoff[b]; j < eoff[b + 1]; ++j) v = fma(ew[j], a[eg[j]], v);
    a[bidx[b]] = v;
}

// ------------------------------------------------------------ restriction
// Coarse interior: FW of the fine interior residual if all 3^d fine
// neighbours are interior, else their FW-weight average over the interior
// ones.  Coarse ghost: the same with ghost/inactive (extended) fine nodes.
template <int D>
__device__ __forceinline__ double restrict_at(const int ic[3], bool interior, const uint8_t *__restrict__ clsf,
                                              const double *__restrict__ rf, const G2 &Gf) {
    // FW weights as integers (1, 2, 4[, 8]) / 4^d: scaling by a power of two
    // is exact, so sum(w_int r) / sum(w_int) equals the weighted mean, and the
    // FW case is sum(w_int r) * 4^-d.
    double fw = 0.0;
    int wsum = 0;
    bool all = true;
#pragma unroll
    for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz)
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
                const int y0 = 2 * ic[0] + ox, y1 = 2 * ic[1] + oy, y2 = 2 * ic[2] + oz;
                if (y0 < 0 || y0 > Gf.N || y1 < 0 || y1 > Gf.N || (D == 3 && (y2 < 0 || y2 > Gf.N))) {
                    all = false;
                    continue;
                }
                const int64_t Y = (int64_t)y0 + (int64_t)y1 * Gf.sy + (int64_t)y2 * Gf.sz;
                const uint8_t c = clsf[Y];
                const bool fam = interior ? (c == CL_INTERIOR) : (c == CL_GHOST || c == CL_INACTIVE);
                if (!fam) {
                    all = false;
                    continue;
                }
                const int wi = (ox == 0 ? 2 : 1) * (oy == 0 ? 2 : 1) * ((D == 3 && oz == 0) ? 2 : 1);
                fw = fma((double)wi, rf[Y], fw);
                wsum += wi;
            }
    if (all) return fw * (D == 3 ? (1.0 / 64.0) : (1.0 / 16.0));
    return wsum > 0 ? fw / (double)wsum : 0.0;
}

template <int D>
__global__ void __launch_bounds__(kT) k_restrict(const Win *__restrict__ win, int64_t nwin, unsigned wblocks,
                                                 const uint32_t *__restrict__ gidx, int64_t ng,
                                                 const uint8_t *__restrict__ clsf, const double *__restrict__ rf,
                                                 double *__restrict__ Fc, double *__restrict__ uc, G2 Gf, G2 Gc) {
    if (blockIdx.x < wblocks) {
        int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (w >= nwin) return;
        const int lane = threadIdx.x & 31;
        const Win W = win[w];
        const int j = W.jk & 0xffffu, k = W.jk >> 16;
        const int i0 = (int)((int64_t)W.base - (int64_t)j * Gc.sy - (int64_t)k * Gc.sz);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = lane + 32 * h;
            if (!((W.mask >> t) & 1ull)) continue;
            const int ic[3] = {i0 + t, j, k};
            const int64_t Xc = (int64_t)W.base + t;
            Fc[Xc] = restrict_at<D>(ic, true, clsf, rf, Gf);
            if (uc) uc[Xc] = 0.0;
        }
        return;
    }
    int64_t g = (int64_t)(blockIdx.x - wblocks) * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const uint32_t Xc = gidx[g];
    const uint32_t n = (uint32_t)Gc.n;
    int ic[3];
    ic[0] = (int)(Xc % n);
    ic[1] = (int)((Xc / n) % n);
    ic[2] = (D == 3) ? (int)(Xc / (n * n)) : 0;
    Fc[Xc] = restrict_at<D>(ic, false, clsf, rf, Gf);
    if (uc) uc[Xc] = 0.0;
}

// ------------------------------------------------------------ prolongation
template <int D>
__device__ __forceinline__ double prolong_at(const int iy[3], const double *__restrict__ ec, const G2 &Gc) {
    int lo[3] = {0, 0, 0}, two[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        lo[a] = iy[a] >> 1;
        two[a] = iy[a] & 1;
    }
    double v = 0.0;
    for (int b2 = 0; b2 <= two[2]; ++b2)
        for (int b1 = 0; b1 <= two[1]; ++b1)
            for (int b0 = 0; b0 <= two[0]; ++b0) {
                const double w = (two[0] ? 0.5 : 1.0) * (two[1] ? 0.5 : 1.0) * (two[2] ? 0.5 : 1.0);
                const int64_t C = (int64_t)(lo[0] + b0) + (int64_t)(lo[1] + b1) * Gc.sy + (int64_t)(lo[2] + b2) * Gc.sz;
                v = fma(w, ec[C], v);
            }
    return v;
}

template <int D>
__global__ void __launch_bounds__(kT) k_prolong(const Win *__restrict__ win, int64_t nwin, unsigned wblocks,
                                                const uint32_t *__restrict__ gidx, int64_t ng,
                                                const double *__restrict__ ec, double *__restrict__ uf, G2 Gf,
                                                G2 Gc) {
    if (blockIdx.x < wblocks) {
        int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (w >= nwin) return;
        const int lane = threadIdx.x & 31;
        const Win W = win[w];
        const int j = W.jk & 0xffffu, k = W.jk >> 16;
        const int i0 = (int)((int64_t)W.base - (int64_t)j * Gf.sy - (int64_t)k * Gf.sz);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = lane + 32 * h;
            if (!((W.mask >> t) & 1ull)) continue;
            const int iy[3] = {i0 + t, j, k};
            const int64_t X = (int64_t)W.base + t;
            uf[X] += prolong_at<D>(iy, ec, Gc);
        }
        return;
    }
    int64_t g = (int64_t)(blockIdx.x - wblocks) * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const uint32_t X = gidx[g];
    const uint32_t n = (uint32_t)Gf.n;
    int iy[3];
    iy[0] = (int)(X % n);
    iy[1] = (int)((X / n) % n);
    iy[2] = (D == 3) ? (int)(X / (n * n)) : 0;
    uf[X] += prolong_at<D>(iy, ec, Gc);
}

// ------------------------------------------------------------ coarsest
__global__ void k_coarse_gather(const uint32_t *__restrict__ act, int64_t nact, const double *__restrict__ r,
                                double *__restrict__ rhs) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nact) rhs[j] = r[act[j]];
}

// u[act[i]] += (A^-1 rhs)_i, one warp per row
__global__ void __launch_bounds__(kT) k_coarse_gemv(const uint32_t *__restrict__ act, int64_t nact,
                                                    const double *__restrict__ Ainv,
                                                    const double *__restrict__ rhs, double *__restrict__ u) {
    int64_t i = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (i >= nact) return;
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int64_t j = lane; j < nact; j += 32) s = fma(Ainv[i * nact + j], rhs[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) u[act[i]] += s;
}

// ------------------------------------------------------------ norms
// Per-block partial sums (sum r_I^2, sum r_G^2, max|r_I|, max|r_G|) in a
// fixed tree order; a single block then reduces the partials in block order.
__global__ void __launch_bounds__(kT) k_norm_partial(const Win *__restrict__ win, int64_t nwin, unsigned wblocks,
                                                     const uint32_t *__restrict__ gidx, int64_t ng,
                                                     const double *__restrict__ r, double *__restrict__ part) {
    __shared__ double sh[4][kT];
    double sI = 0.0, sG = 0.0, mI = 0.0, mG = 0.0;
    if (blockIdx.x < wblocks) {
        int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (w < nwin) {
            const int lane = threadIdx.x & 31;
            const Win W = win[w];
            for (int h = 0; h < 2; ++h) {
                const int t = lane + 32 * h;
                if ((W.mask >> t) & 1ull) {
                    const double v = r[(int64_t)W.base + t];
                    sI = fma(v, v, sI);
                    mI = fmax(mI, fabs(v));
                }
            }
        }
    } else {
        int64_t g = (int64_t)(blockIdx.x - wblocks) * blockDim.x + threadIdx.x;
        if (g < ng) {
            const double v = r[gidx[g]];
            sG = v * v;
            mG = fabs(v);
        }
    }
    sh[0][threadIdx.x] = sI;
    sh[1][threadIdx.x] = sG;
    sh[2][threadIdx.x] = mI;
    sh[3][threadIdx.x] = mG;
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + s]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) part[(int64_t)blockIdx.x * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(1024) k_norm_final(const double *__restrict__ part, int64_t nparts,
                                                     double *__restrict__ out) {
    __shared__ double sh[4][1024];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < nparts; i += blockDim.x) {
        a[0] += part[i * 4 + 0];
        a[1] += part[i * 4 + 1];
        a[2] = fmax(a[2], part[i * 4 + 2]);
        a[3] = fmax(a[3], part[i * 4 + 3]);
    }
    for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = a[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + s]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sqrt(sh[0][0]);
        out[1] = sqrt(sh[1][0]);
        out[2] = sh[2][0];
        out[3] = sh[3][0];
    }
}

// ------------------------------------------------------------ data movement
__global__ void __launch_bounds__(kT) k_copy_active(const Win *__restrict__ win, int64_t nwin, unsigned wblocks,
                                                    const uint32_t *__restrict__ gidx, int64_t ng, unsigned gblocks,
                                                    const uint32_t *__restrict__ box, int64_t nbox,
                                                    const double *__restrict__ src, double *__restrict__ dst) {
    if (blockIdx.x < wblocks) {
        int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (w >= nwin) return;
        const int lane = threadIdx.x & 31;
        const Win W = win[w];
        for (int h = 0; h < 2; ++h) {
            const int t = lane + 32 * h;
            if ((W.mask >> t) & 1ull) dst[(int64_t)W.base + t] = src[(int64_t)W.base + t];
        }
        return;
    }
    if (blockIdx.x < wblocks + gblocks) {
        int64_t g = (int64_t)(blockIdx.x - wblocks) * blockDim.x + threadIdx.x;
        if (g < ng) dst[gidx[g]] = src[gidx[g]];
        return;
    }
    int64_t b = (int64_t)(blockIdx.x - wblocks - gblocks) * blockDim.x + threadIdx.x;
    if (b < nbox) dst[box[b]] = src[box[b]];
}

__global__ void k_scatter_ghosts(const uint32_t *__restrict__ gidx, int64_t ng, const double *__restrict__ g,
                                 double *__restrict__ F) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ng) F[gidx[i]] = g[i];
}

__global__ void __launch_bounds__(kT) k_set_interior(const Win *__restrict__ win, int64_t nwin,
                                                     const double *__restrict__ f, double *__restrict__ F) {
    int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= nwin) return;
    const int lane = threadIdx.x & 31;
    const Win W = win[w];
    for (int h = 0; h < 2; ++h) {
        const int t = lane + 32 * h;
        if ((W.mask >> t) & 1ull) F[(int64_t)W.base + t] = f ? f[(int64_t)W.base + t] : 0.0;
    }
}

}  // namespace

// ------------------------------------------------------------ host wrappers

void smooth(Handle &H, Level &L, double *u, const double *F, int nsteps) {
    const G2 G = g2_of(L);
    for (int s = 0; s < nsteps; ++s) {
        for (int c = 0; c < 2; ++c) {
            profile_mark(H, L);
            if (L.d == 3) LAUNCH(k_smooth<3>, wblk(L.nwin), kT, L.win, L.nwin, u, F, G, c);
            else LAUNCH(k_smooth<2>, wblk(L.nwin), kT, L.win, L.nwin, u, F, G, c);
            profile_mark(H, L);
        }
        if (L.d == 3)
            LAUNCH(k_ghost_relax<3>, nblk(L.ng, 128), 128, L.gidx, L.gcode, L.gxi, L.gdt, L.ng, u, F, L.gtmp, G);
        else
            LAUNCH(k_ghost_relax<2>, nblk(L.ng, 128), 128, L.gidx, L.gcode, L.gxi, L.gdt, L.ng, u, F, L.gtmp, G);
        LAUNCH(k_ghost_scatter, nblk(L.ng, 256), 256, L.gidx, L.ng, L.gtmp, u);
    }
}

void residual(Handle &H, Level &L, const double *u, const double *F, double *r) {
    const G2 G = g2_of(L);
    const unsigned wb = wblk(L.nwin);
    const unsigned grid = wb + nblk(L.ng, kT);
    if (L.d == 3) LAUNCH(k_residual<3>, grid, kT, L.win, L.nwin, wb, L.gidx, L.gcode, L.gxi, L.ng, u, F, r, G);
    else LAUNCH(k_residual<2>, grid, kT, L.win, L.nwin, wb, L.gidx, L.gcode, L.gxi, L.ng, u, F, r, G);
}

void extend(Handle &H, Level &L, double *a) {
    if (L.nb == 0) return;
    if (L.eoff) {
        LAUNCH(k_extend_csr, nblk(L.nb, 256), 256, L.bidx, L.eoff, L.eg, L.ew, L.nb, a);
        return;
    }
    const int K = std::max(H.o.ext_sweeps, 1);
    double *b0 = L.bbuf, *b1 = L.bbuf + L.nb;
    const double *in = nullptr;
    for (int k = 0; k < K; ++k) {
        const int last = (k == K - 1);
        double *out = (k % 2 == 0) ? b0 : b1;
        LAUNCH(k_extend, nblk(L.nb, 256), 256, L.bidx, L.bref, L.bw, L.nb, L.d, a, in, out, last);
        in = out;
    }
}

void restrict_to(Handle &H, Level &Lf, Level &Lc, const double *rf, double *Fc, double *uc_zero) {
    const G2 Gf = g2_of(Lf), Gc = g2_of(Lc);
    const unsigned wb = wblk(Lc.nwin);
    const unsigned grid = wb + nblk(Lc.ng, kT);
    if (Lf.d == 3)
        LAUNCH(k_restrict<3>, grid, kT, Lc.win, Lc.nwin, wb, Lc.gidx, Lc.ng, Lf.cls, rf, Fc, uc_zero, Gf, Gc);
    else
        LAUNCH(k_restrict<2>, grid, kT, Lc.win, Lc.nwin, wb, Lc.gidx, Lc.ng, Lf.cls, rf, Fc, uc_zero, Gf, Gc);
}

void prolong(Handle &H, Level &Lf, Level &Lc, const double *ec, double *uf) {
    const G2 Gf = g2_of(Lf), Gc = g2_of(Lc);
    const unsigned wb = wblk(Lf.nwin);
    const unsigned grid = wb + nblk(Lf.ng, kT);
    if (Lf.d == 3) LAUNCH(k_prolong<3>, grid, kT, Lf.win, Lf.nwin, wb, Lf.gidx, Lf.ng, ec, uf, Gf, Gc);
    else LAUNCH(k_prolong<2>, grid, kT, Lf.win, Lf.nwin, wb, Lf.gidx, Lf.ng, ec, uf, Gf, Gc);
}

void coarsest_correct(Handle &H, Level &L, double *u, const double *F) {
    residual(H, L, u, F, L.r);
    LAUNCH(k_coarse_gather, nblk(L.nact, 256), 256, L.act, L.nact, L.r, L.crhs);
    LAUNCH(k_coarse_gemv, wblk(L.nact), kT, L.act, L.nact, L.Ainv, L.crhs, u);
}

void norms(Handle &H, Level &L, const double *r, double *out4) {
    const unsigned wb = wblk(L.nwin);
    const unsigned grid = wb + nblk(L.ng, kT);
    LAUNCH(k_norm_partial, grid, kT, L.win, L.nwin, wb, L.gidx, L.ng, r, H.npart);
    LAUNCH(k_norm_final, 1u, 1024, H.npart, (int64_t)grid, out4);
}

// V(nu1, nu2) cycle from level l down (Sec. 2.1 with gamma = 1); u is the
// level's unknown (finest: the working copy, coarse: the correction).
void vcycle_enqueue(Handle &H, int l, double *u) {
    Level &A = H.L[l];
    if (l == (int)H.L.size() - 1) {
        coarsest_correct(H, A, u, A.F);
        return;
    }
    Level &B = H.L[l + 1];
    smooth(H, A, u, A.F, H.o.nu1);
    residual(H, A, u, A.F, A.r);
    extend(H, A, A.r);
    restrict_to(H, A, B, A.r, B.F, B.u);
    vcycle_enqueue(H, l + 1, B.u);
    extend(H, B, B.u);
    prolong(H, A, B, B.u, u);
    smooth(H, A, u, A.F, H.o.nu2);
}

void copy_active(Handle &H, const double *src, double *dst, bool with_boxdir) {
    Level &L = H.L[0];
    const unsigned wb = wblk(L.nwin), gb = nblk(L.ng, kT);
    const int64_t nbox = with_boxdir ? L.nbox : 0;
    const unsigned grid = wb + gb + nblk(nbox, kT);
    LAUNCH(k_copy_active, grid, kT, L.win, L.nwin, wb, L.gidx, L.ng, gb, L.boxidx, nbox, src, dst);
}

void scatter_ghost_values(Handle &H, Level &L, const double *g, double *F) {
    LAUNCH(k_scatter_ghosts, nblk(L.ng, 256), 256, L.gidx, L.ng, g, F);
}

void set_interior_rhs(Handle &H, Level &L, const double *f, double *F) {
    LAUNCH(k_set_interior, wblk(L.nwin), kT, L.win, L.nwin, f, F);
}

}  // namespace bcmg
