// Multigrid cycle kernels of the GB300 BCMG library (arXiv 2207.14208).
//
// Interior work runs over the compacted 64-node windows (one warp per
// window, coalesced x-rows, no class reads); ghost and band work over their
// compacted lists.  Every cycle kernel is templated on the value type: FP64
// for the plain cycle, FP32 for the inner cycle of the mixed-precision
// refinement (whose outer residual and update stay FP64).  None of them is a
// dense contraction, so no tensor-core path is used.
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

template <typename K, typename... A>
void launch(Handle &H, const char *name, K kern, unsigned grid, unsigned block, A... args) {
    if (grid == 0) return;
    kern<<<grid, block, 0, H.st>>>(args...);
    check_cuda(cudaGetLastError(), name);
    count_launch(H);
}

// quadratic / linear / constant Lagrange basis on local nodes 0, 1, 2
// (eq. coeff: c_0, c_-1, c_-2 at xi = theta)
template <typename T>
__device__ __forceinline__ void lagrange(int q, T xi, T w[3]) {
    if (q == 2) {
        w[0] = (T(1) - xi) * (T(2) - xi) * T(0.5);
        w[1] = xi * (T(2) - xi);
        w[2] = xi * (xi - T(1)) * T(0.5);
    } else if (q == 1) {
        w[0] = T(1) - xi;
        w[1] = xi;
        w[2] = T(0);
    } else {
        w[0] = T(1);
        w[1] = T(0);
        w[2] = T(0);
    }
}

// B u~ at a ghost: the (tri/bi)quadratic interpolant on ST_G at Q (eq. BCh).
// Fully unrolled with compile-time stencil offsets (weights stay in
// registers); nodes beyond an axis' degree are never loaded.
template <int D, typename T>
__device__ __forceinline__ T ghost_B(int64_t X, uint16_t code, const double *__restrict__ gxi, int64_t ng,
                                     int64_t g, const T *u, const G2 &G) {
    const int qx = (code >> 3) & 3, qy = (code >> 5) & 3, qz = (D == 3) ? ((code >> 7) & 3) : 0;
    const int64_t ox = (code & 1) ? 1 : -1;
    const int64_t oy = (code & 2) ? G.sy : -G.sy;
    const int64_t oz = (D == 3) ? ((code & 4) ? G.sz : -G.sz) : 0;
    T wx[3], wy[3], wz[3] = {T(1), T(0), T(0)};
    lagrange<T>(qx, (T)gxi[g], wx);
    lagrange<T>(qy, (T)gxi[ng + g], wy);
    if (D == 3) lagrange<T>(qz, (T)gxi[2 * ng + g], wz);
    T B = T(0);
#pragma unroll
    for (int o2 = 0; o2 < (D == 3 ? 3 : 1); ++o2) {
        if (o2 > qz) break;
#pragma unroll
        for (int o1 = 0; o1 < 3; ++o1) {
            if (o1 > qy) break;
            const T wyz = wz[o2] * wy[o1];
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

template <int D, typename T>
__device__ __forceinline__ T nbr_sum(const T *u, int64_t X, const G2 &G) {
    T s = (u[X - 1] + u[X + 1]) + (u[X - G.sy] + u[X + G.sy]);
    if (D == 3) s += u[X - G.sz] + u[X + G.sz];
    return s;
}

// ------------------------------------------------------------ smoothing
// One colour of red-black Gauss-Seidel on interior nodes (eq. GSLEX_2D in
// red-black order): u_X = (sum of 2d neighbours + h^2 F_X) / (2d).
template <int D, typename T>
__global__ void __launch_bounds__(kT) k_smooth(const Win *__restrict__ win, int64_t nwin, T *u,
                                               const T *__restrict__ F, G2 G, int color) {
    int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= nwin) return;
    const int lane = threadIdx.x & 31;
    const Win W = win[w];
    const int par = ((W.jk & 0xffffu) + (W.jk >> 16)) & 1;
    const int t = 2 * lane + ((color ^ par) & 1);
    if (!((W.mask >> t) & 1ull)) return;
    const int64_t X = (int64_t)W.base + t;
    const T s = nbr_sum<D, T>(u, X, G);
    u[X] = fma((T)G.h2, F[X], s) * (T)G.inv2d;
}

// Fictitious-time relaxation of all ghosts from the same u (eq. rel with
// eq. DtauOptTheta; the ghost block of P is diag(1/Delta tau)): new values go
// to tmp, then k_ghost_scatter writes them.
template <int D, typename T>
__global__ void k_ghost_relax(const uint32_t *__restrict__ gidx, const uint16_t *__restrict__ gcode,
                              const double *__restrict__ gxi, const double *__restrict__ gdt, int64_t ng,
                              const T *u, const T *__restrict__ F, T *__restrict__ tmp, G2 G) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int64_t X = gidx[g];
    const T B = ghost_B<D, T>(X, gcode[g], gxi, ng, g, u, G);
    tmp[g] = fma((T)gdt[g], F[X] - B, u[X]);
}

template <typename T>
__global__ void k_ghost_scatter(const uint32_t *__restrict__ gidx, int64_t ng, const T *__restrict__ tmp,
                                T *__restrict__ u) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    u[gidx[g]] = tmp[g];
}

// ------------------------------------------------------------ residual
// r = F - A u on interior rows (eq. Laph) and ghost rows (eq. BCh).
template <int D, typename T>
__global__ void __launch_bounds__(kT) k_residual(const Win *__restrict__ win, int64_t nwin, unsigned wblocks,
                                                 const uint32_t *__restrict__ gidx,
                                                 const uint16_t *__restrict__ gcode,
                                                 const double *__restrict__ gxi, int64_t ng,
                                                 const T *__restrict__ u, const T *__restrict__ F,
                                                 T *__restrict__ r, G2 G) {
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
            const T s = nbr_sum<D, T>(u, X, G);
            r[X] = F[X] - (T(2 * D) * u[X] - s) * (T)G.ih2;
        }
        return;
    }
    int64_t g = (int64_t)(blockIdx.x - wblocks) * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int64_t X = gidx[g];
    r[X] = F[X] - ghost_B<D, T>(X, gcode[g], gxi, ng, g, u, G);
}

// ------------------------------------------------------------ band extension
// One explicit pseudo-time sweep of dr/dsigma + dr/dn = 0 with upwind
// differences at the largest stable step: each band value becomes the
// normalised |n_a|-weighted mean of its upwind ghost / band sources.
template <typename T>
__global__ void k_extend(const uint32_t *__restrict__ bidx, const int32_t *__restrict__ bref,
                         const double *__restrict__ bw, int64_t nb, int d, T *a, const T *__restrict__ in,
                         T *__restrict__ out, int last) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    T v = T(0);
    for (int ax = 0; ax < d; ++ax) {
        const int32_t ref = bref[(int64_t)ax * nb + b];
        if (ref == kNoRef) continue;
        T s;
        if (ref < 0) s = a[-(int64_t)ref - 1];
        else s = in ? in[ref] : T(0);
        v = fma((T)bw[(int64_t)ax * nb + b], s, v);
    }
    if (last) a[bidx[b]] = v;
    else out[b] = v;
}

// All K sweeps at once: band value = sum over the precomputed (ghost, weight)
// terms of the band node (the expansion of the sweeps started from zero),
// ELL layout with the terms of one slot contiguous across band nodes.
template <typename T>
__global__ void k_extend_ell(const uint32_t *__restrict__ bidx, const uint8_t *__restrict__ ecnt,
                             const uint32_t *__restrict__ eg, const double *__restrict__ ew, int64_t nb, T *a) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    T v = T(0);
    const int c = ecnt[b];
    for (int k = 0; k < c; ++k) v = fma((T)ew[(int64_t)k * nb + b], a[eg[(int64_t)k * nb + b]], v);
    a[bidx[b]] = v;
}

// ------------------------------------------------------------ restriction
// Coarse interior: FW of the fine interior residual if all 3^d fine
// neighbours are interior, else their FW-weight average over the interior
// ones.  Coarse ghost: the same with ghost/inactive (extended) fine nodes.
template <int D, typename T>
__device__ __forceinline__ T restrict_at(const int ic[3], bool interior, const uint8_t *__restrict__ clsf,
                                         const T *__restrict__ rf, const G2 &Gf) {
    // FW weights as integers (1, 2, 4[, 8]) / 4^d: scaling by a power of two
    // is exact, so sum(w_int r) / sum(w_int) equals the weighted mean, and the
    // FW case is sum(w_int r) * 4^-d.
    T fw = T(0);
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
                fw = fma((T)wi, rf[Y], fw);
                wsum += wi;
            }
    if (all) return fw * (D == 3 ? T(1.0 / 64.0) : T(1.0 / 16.0));
    return wsum > 0 ? fw / (T)wsum : T(0);
}

template <int D, typename T>
__global__ void __launch_bounds__(kT) k_restrict(const Win *__restrict__ win, int64_t nwin, unsigned wblocks,
                                                 const uint32_t *__restrict__ gidx, int64_t ng,
                                                 const uint8_t *__restrict__ clsf, const T *__restrict__ rf,
                                                 T *__restrict__ Fc, T *__restrict__ uc, G2 Gf, G2 Gc) {
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
            Fc[Xc] = restrict_at<D, T>(ic, true, clsf, rf, Gf);
            if (uc) uc[Xc] = T(0);
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
    Fc[Xc] = restrict_at<D, T>(ic, false, clsf, rf, Gf);
    if (uc) uc[Xc] = T(0);
}

// ------------------------------------------------------------ prolongation
template <int D, typename T>
__device__ __forceinline__ T prolong_at(const int iy[3], const T *__restrict__ ec, const G2 &Gc) {
    int lo[3] = {0, 0, 0}, two[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        lo[a] = iy[a] >> 1;
        two[a] = iy[a] & 1;
    }
    T v = T(0);
    for (int b2 = 0; b2 <= two[2]; ++b2)
        for (int b1 = 0; b1 <= two[1]; ++b1)
            for (int b0 = 0; b0 <= two[0]; ++b0) {
                const T w = (two[0] ? T(0.5) : T(1)) * (two[1] ? T(0.5) : T(1)) * (two[2] ? T(0.5) : T(1));
                const int64_t C = (int64_t)(lo[0] + b0) + (int64_t)(lo[1] + b1) * Gc.sy + (int64_t)(lo[2] + b2) * Gc.sz;
                v = fma(w, ec[C], v);
            }
    return v;
}

template <int D, typename T>
__global__ void __launch_bounds__(kT) k_prolong(const Win *__restrict__ win, int64_t nwin, unsigned wblocks,
                                                const uint32_t *__restrict__ gidx, int64_t ng,
                                                const T *__restrict__ ec, T *__restrict__ uf, G2 Gf, G2 Gc) {
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
            uf[X] += prolong_at<D, T>(iy, ec, Gc);
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
    uf[X] += prolong_at<D, T>(iy, ec, Gc);
}

// ------------------------------------------------------------ coarsest
template <typename T>
__global__ void k_coarse_gather(const uint32_t *__restrict__ act, int64_t nact, const T *__restrict__ r,
                                double *__restrict__ rhs) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nact) rhs[j] = (double)r[act[j]];
}

// u[act[i]] += (A^-1 rhs)_i, one warp per row (FP64 accumulation)
template <typename T>
__global__ void __launch_bounds__(kT) k_coarse_gemv(const uint32_t *__restrict__ act, int64_t nact,
                                                    const double *__restrict__ Ainv,
                                                    const double *__restrict__ rhs, T *__restrict__ u) {
    int64_t i = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (i >= nact) return;
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int64_t j = lane; j < nact; j += 32) s = fma(Ainv[i * nact + j], rhs[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) u[act[i]] += (T)s;
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

// ------------------------------------------------------------ mixed precision
// Start of one refinement step on the finest level: the FP32 right-hand side
// is the FP64 residual rounded to FP32, the FP32 correction starts at zero.
__global__ void __launch_bounds__(kT) k_ir_begin(const Win *__restrict__ win, int64_t nwin, unsigned wblocks,
                                                 const uint32_t *__restrict__ gidx, int64_t ng,
                                                 const double *__restrict__ r, float *__restrict__ F32,
                                                 float *__restrict__ e32) {
    if (blockIdx.x < wblocks) {
        int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (w >= nwin) return;
        const int lane = threadIdx.x & 31;
        const Win W = win[w];
        for (int h = 0; h < 2; ++h) {
            const int t = lane + 32 * h;
            if ((W.mask >> t) & 1ull) {
                const int64_t X = (int64_t)W.base + t;
                F32[X] = (float)r[X];
                e32[X] = 0.0f;
            }
        }
        return;
    }
    int64_t g = (int64_t)(blockIdx.x - wblocks) * blockDim.x + threadIdx.x;
    if (g < ng) {
        const int64_t X = gidx[g];
        F32[X] = (float)r[X];
        e32[X] = 0.0f;
    }
}

// End of a refinement step: u += e on interior and ghost nodes (FP64).
__global__ void __launch_bounds__(kT) k_ir_update(const Win *__restrict__ win, int64_t nwin, unsigned wblocks,
                                                  const uint32_t *__restrict__ gidx, int64_t ng,
                                                  const float *__restrict__ e32, double *__restrict__ u) {
    if (blockIdx.x < wblocks) {
        int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (w >= nwin) return;
        const int lane = threadIdx.x & 31;
        const Win W = win[w];
        for (int h = 0; h < 2; ++h) {
            const int t = lane + 32 * h;
            if ((W.mask >> t) & 1ull) {
                const int64_t X = (int64_t)W.base + t;
                u[X] += (double)e32[X];
            }
        }
        return;
    }
    int64_t g = (int64_t)(blockIdx.x - wblocks) * blockDim.x + threadIdx.x;
    if (g < ng) {
        const int64_t X = gidx[g];
        u[X] += (double)e32[X];
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

// level arrays of one precision
template <typename T> struct Arr;
template <> struct Arr<double> {
    static double *u(Level &L) { return L.u; }
    static double *F(Level &L) { return L.F; }
    static double *r(Level &L) { return L.r; }
    static double *gtmp(Level &L) { return L.gtmp; }
    static double *bbuf(Level &L) { return L.bbuf; }
};
template <> struct Arr<float> {
    static float *u(Level &L) { return L.u32; }
    static float *F(Level &L) { return L.F32; }
    static float *r(Level &L) { return L.r32; }
    static float *gtmp(Level &L) { return L.gtmp32; }
    static float *bbuf(Level &L) { return L.bbuf32; }
};

template <typename T>
void vcycle_t(Handle &H, int l, T *u) {
    Level &A = H.L[l];
    if (l == (int)H.L.size() - 1) {
        coarsest_correct<T>(H, A, u, Arr<T>::F(A));
        return;
    }
    Level &B = H.L[l + 1];
    smooth<T>(H, A, u, Arr<T>::F(A), H.o.nu1);
    residual<T>(H, A, u, Arr<T>::F(A), Arr<T>::r(A));
    extend<T>(H, A, Arr<T>::r(A));
    restrict_to<T>(H, A, B, Arr<T>::r(A), Arr<T>::F(B), Arr<T>::u(B));
    vcycle_t<T>(H, l + 1, Arr<T>::u(B));
    extend<T>(H, B, Arr<T>::u(B));
    prolong<T>(H, A, B, Arr<T>::u(B), u);
    smooth<T>(H, A, u, Arr<T>::F(A), H.o.nu2);
}

}  // namespace

// ------------------------------------------------------------ host wrappers

template <typename T>
void smooth(Handle &H, Level &L, T *u, const T *F, int nsteps) {
    const G2 G = g2_of(L);
    T *tmp = Arr<T>::gtmp(L);
    // the timed sweeps are the finest-level ones of the solve's working precision
    const bool prof = (sizeof(T) == 8) == (H.o.precision == BCMG_PREC_FP64);
    for (int s = 0; s < nsteps; ++s) {
        for (int c = 0; c < 2; ++c) {
            if (prof) profile_mark(H, L);
            if (L.d == 3) launch(H, "k_smooth", k_smooth<3, T>, wblk(L.nwin), kT, L.win, L.nwin, u, F, G, c);
            else launch(H, "k_smooth", k_smooth<2, T>, wblk(L.nwin), kT, L.win, L.nwin, u, F, G, c);
            if (prof) profile_mark(H, L);
        }
        if (L.d == 3)
            launch(H, "k_ghost_relax", k_ghost_relax<3, T>, nblk(L.ng, 128), 128, L.gidx, L.gcode, L.gxi, L.gdt,
                   L.ng, (const T *)u, F, tmp, G);
        else
            launch(H, "k_ghost_relax", k_ghost_relax<2, T>, nblk(L.ng, 128), 128, L.gidx, L.gcode, L.gxi, L.gdt,
                   L.ng, (const T *)u, F, tmp, G);
        launch(H, "k_ghost_scatter", k_ghost_scatter<T>, nblk(L.ng, 256), 256, L.gidx, L.ng, (const T *)tmp, u);
    }
}

template <typename T>
void residual(Handle &H, Level &L, const T *u, const T *F, T *r) {
    const G2 G = g2_of(L);
    const unsigned wb = wblk(L.nwin);
    const unsigned grid = wb + nblk(L.ng, kT);
    if (L.d == 3)
        launch(H, "k_residual", k_residual<3, T>, grid, kT, L.win, L.nwin, wb, L.gidx, L.gcode, L.gxi, L.ng, u, F,
               r, G);
    else
        launch(H, "k_residual", k_residual<2, T>, grid, kT, L.win, L.nwin, wb, L.gidx, L.gcode, L.gxi, L.ng, u, F,
               r, G);
}

template <typename T>
void extend(Handle &H, Level &L, T *a) {
    if (L.nb == 0) return;
    if (L.ecnt) {
        launch(H, "k_extend_ell", k_extend_ell<T>, nblk(L.nb, 256), 256, (const uint32_t *)L.bidx,
               (const uint8_t *)L.ecnt, (const uint32_t *)L.eg, (const double *)L.ew, L.nb, a);
        return;
    }
    const int K = std::max(H.o.ext_sweeps, 1);
    T *b0 = Arr<T>::bbuf(L), *b1 = Arr<T>::bbuf(L) + L.nb;
    const T *in = nullptr;
    for (int k = 0; k < K; ++k) {
        const int last = (k == K - 1);
        T *out = (k % 2 == 0) ? b0 : b1;
        launch(H, "k_extend", k_extend<T>, nblk(L.nb, 256), 256, L.bidx, L.bref, L.bw, L.nb, L.d, a, in, out, last);
        in = out;
    }
}

template <typename T>
void restrict_to(Handle &H, Level &Lf, Level &Lc, const T *rf, T *Fc, T *uc_zero) {
    const G2 Gf = g2_of(Lf), Gc = g2_of(Lc);
    const unsigned wb = wblk(Lc.nwin);
    const unsigned grid = wb + nblk(Lc.ng, kT);
    if (Lf.d == 3)
        launch(H, "k_restrict", k_restrict<3, T>, grid, kT, Lc.win, Lc.nwin, wb, Lc.gidx, Lc.ng,
               (const uint8_t *)Lf.cls, rf, Fc, uc_zero, Gf, Gc);
    else
        launch(H, "k_restrict", k_restrict<2, T>, grid, kT, Lc.win, Lc.nwin, wb, Lc.gidx, Lc.ng,
               (const uint8_t *)Lf.cls, rf, Fc, uc_zero, Gf, Gc);
}

template <typename T>
void prolong(Handle &H, Level &Lf, Level &Lc, const T *ec, T *uf) {
    const G2 Gf = g2_of(Lf), Gc = g2_of(Lc);
    const unsigned wb = wblk(Lf.nwin);
    const unsigned grid = wb + nblk(Lf.ng, kT);
    if (Lf.d == 3)
        launch(H, "k_prolong", k_prolong<3, T>, grid, kT, Lf.win, Lf.nwin, wb, Lf.gidx, Lf.ng, ec, uf, Gf, Gc);
    else
        launch(H, "k_prolong", k_prolong<2, T>, grid, kT, Lf.win, Lf.nwin, wb, Lf.gidx, Lf.ng, ec, uf, Gf, Gc);
}

template <typename T>
void coarsest_correct(Handle &H, Level &L, T *u, const T *F) {
    residual<T>(H, L, u, F, Arr<T>::r(L));
    launch(H, "k_coarse_gather", k_coarse_gather<T>, nblk(L.nact, 256), 256, L.act, L.nact,
           (const T *)Arr<T>::r(L), L.crhs);
    launch(H, "k_coarse_gemv", k_coarse_gemv<T>, wblk(L.nact), kT, L.act, L.nact, (const double *)L.Ainv,
           (const double *)L.crhs, u);
}

void norms(Handle &H, Level &L, const double *r, double *out4) {
    const unsigned wb = wblk(L.nwin);
    const unsigned grid = wb + nblk(L.ng, kT);
    launch(H, "k_norm_partial", k_norm_partial, grid, kT, L.win, L.nwin, wb, L.gidx, L.ng, r, H.npart);
    launch(H, "k_norm_final", k_norm_final, 1u, 1024u, (const double *)H.npart, (int64_t)grid, out4);
}

// V(nu1, nu2) cycle from level l down (Sec. 2.1 with gamma = 1); u is the
// level's unknown (finest: the working copy, coarse: the correction).
void vcycle_enqueue(Handle &H, int l, double *u) { vcycle_t<double>(H, l, u); }

void mixed_step_enqueue(Handle &H, double *u) {
    Level &L = H.L[0];
    const unsigned wb = wblk(L.nwin);
    const unsigned grid = wb + nblk(L.ng, kT);
    launch(H, "k_ir_begin", k_ir_begin, grid, kT, L.win, L.nwin, wb, L.gidx, L.ng, (const double *)L.r, L.F32,
           L.u32);
    vcycle_t<float>(H, 0, L.u32);
    launch(H, "k_ir_update", k_ir_update, grid, kT, L.win, L.nwin, wb, L.gidx, L.ng, (const float *)L.u32, u);
}

void copy_active(Handle &H, const double *src, double *dst, bool with_boxdir) {
    Level &L = H.L[0];
    const unsigned wb = wblk(L.nwin), gb = nblk(L.ng, kT);
    const int64_t nbox = with_boxdir ? L.nbox : 0;
    const unsigned grid = wb + gb + nblk(nbox, kT);
    launch(H, "k_copy_active", k_copy_active, grid, kT, L.win, L.nwin, wb, L.gidx, L.ng, gb,
           (const uint32_t *)L.boxidx, nbox, src, dst);
}

void scatter_ghost_values(Handle &H, Level &L, const double *g, double *F) {
    launch(H, "k_scatter_ghosts", k_scatter_ghosts, nblk(L.ng, 256), 256, L.gidx, L.ng, g, F);
}

void set_interior_rhs(Handle &H, Level &L, const double *f, double *F) {
    launch(H, "k_set_interior", k_set_interior, wblk(L.nwin), kT, L.win, L.nwin, f, F);
}

template void smooth<double>(Handle &, Level &, double *, const double *, int);
template void residual<double>(Handle &, Level &, const double *, const double *, double *);
template void extend<double>(Handle &, Level &, double *);
template void restrict_to<double>(Handle &, Level &, Level &, const double *, double *, double *);
template void prolong<double>(Handle &, Level &, Level &, const double *, double *);
template void coarsest_correct<double>(Handle &, Level &, double *, const double *);
template void smooth<float>(Handle &, Level &, float *, const float *, int);
template void residual<float>(Handle &, Level &, const float *, const float *, float *);
template void extend<float>(Handle &, Level &, float *);
template void restrict_to<float>(Handle &, Level &, Level &, const float *, float *, float *);
template void prolong<float>(Handle &, Level &, Level &, const float *, float *);
template void coarsest_correct<float>(Handle &, Level &, float *, const float *);

}  // namespace bcmg
