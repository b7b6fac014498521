// Hierarchy set-up on the GPU: per-level node classes, interior windows,
// ghost projection / stencil / Delta tau, band lists and the coarsest-level
// inverse (arXiv 2207.14208, Sec. 3.3 geometry, Sec. 3.2-4.1 BLFA).
//
// The geometric decisions (classes, normals, the bisection for eta, the
// stencil directions and fall-backs, band membership) use explicitly rounded
// IEEE operations so that they do not depend on FMA contraction.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "bcmg_internal.cuh"

namespace bcmg {

namespace {

struct Geo {
    int d, N, n;
    int64_t st[3];
    double h;
};

Geo geo_of(const Level &L) {
    Geo g;
    g.d = L.d;
    g.N = L.N;
    g.n = L.n;
    for (int a = 0; a < 3; ++a) g.st[a] = L.st[a];
    g.h = L.h;
    return g;
}

__device__ __forceinline__ void decode(const Geo &G, int64_t lin, int ix[3]) {
    uint64_t v = (uint64_t)lin;
    ix[0] = ix[1] = ix[2] = 0;
    for (int a = 0; a < G.d; ++a) {
        ix[a] = (int)(v % (uint64_t)G.n);
        v /= (uint64_t)G.n;
    }
}

__device__ __forceinline__ bool in_grid(const Geo &G, const int ix[3]) {
    for (int a = 0; a < G.d; ++a)
        if (ix[a] < 0 || ix[a] > G.N) return false;
    return true;
}

__device__ __forceinline__ int64_t lin_of(const Geo &G, const int ix[3]) {
    int64_t s = 0;
    for (int a = 0; a < G.d; ++a) s += (int64_t)ix[a] * G.st[a];
    return s;
}

// ---------------------------------------------------------------- compaction
constexpr int kCompactThreads = 256;
constexpr int kCompactPerThread = 16;
constexpr int kCompactTile = kCompactThreads * kCompactPerThread;

__global__ void k_count(const uint8_t *__restrict__ flags, int64_t n, int64_t *__restrict__ counts) {
    __shared__ int64_t red[kCompactThreads];
    int64_t base = (int64_t)blockIdx.x * kCompactTile + (int64_t)threadIdx.x * kCompactPerThread;
    int64_t c = 0;
    for (int i = 0; i < kCompactPerThread; ++i)
        if (base + i < n) c += flags[base + i] ? 1 : 0;
    red[threadIdx.x] = c;
    __syncthreads();
    for (int s = kCompactThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[blockIdx.x] = red[0];
}

__global__ void k_scatter(const uint8_t *__restrict__ flags, int64_t n, const int64_t *__restrict__ offs,
                          uint32_t *__restrict__ out) {
    __shared__ int64_t sc[kCompactThreads];
    int64_t base = (int64_t)blockIdx.x * kCompactTile + (int64_t)threadIdx.x * kCompactPerThread;
    int64_t c = 0;
    for (int i = 0; i < kCompactPerThread; ++i)
        if (base + i < n) c += flags[base + i] ? 1 : 0;
    sc[threadIdx.x] = c;
    __syncthreads();
    // inclusive Hillis-Steele scan over the block (deterministic)
    for (int s = 1; s < kCompactThreads; s <<= 1) {
        int64_t v = (threadIdx.x >= s) ? sc[threadIdx.x - s] : 0;
        __syncthreads();
        sc[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t pos = offs[blockIdx.x] + sc[threadIdx.x] - c;
    for (int i = 0; i < kCompactPerThread; ++i)
        if (base + i < n && flags[base + i]) out[pos++] = (uint32_t)(base + i);
}

// ---------------------------------------------------------------- classes
__global__ void k_inject(const double *__restrict__ phif, Geo Gf, Geo Gc, double *__restrict__ phic) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nn = 1;
    for (int a = 0; a < Gc.d; ++a) nn *= Gc.n;
    if (c >= nn) return;
    int ic[3];
    decode(Gc, c, ic);
    int iy[3] = {2 * ic[0], 2 * ic[1], 2 * ic[2]};
    phic[c] = phif[lin_of(Gf, iy)];
}

__device__ __forceinline__ bool interior_at(const Geo &G, const double *phi, const int ix[3]) {
    for (int a = 0; a < G.d; ++a)
        if (ix[a] == 0 || ix[a] == G.N) return false;
    return phi[lin_of(G, ix)] < 0.0;
}

__global__ void k_classify(const double *__restrict__ phi, Geo G, int64_t nn, uint8_t *__restrict__ cls) {
    int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (lin >= nn) return;
    int ix[3];
    decode(G, lin, ix);
    bool edge = false;
    for (int a = 0; a < G.d; ++a)
        if (ix[a] == 0 || ix[a] == G.N) edge = true;
    uint8_t c;
    if (phi[lin] < 0.0) {
        c = edge ? CL_BOXDIR : CL_INTERIOR;
    } else {
        c = CL_INACTIVE;
        for (int a = 0; a < G.d; ++a)
            for (int dir = -1; dir <= 1; dir += 2) {
                int iy[3] = {ix[0], ix[1], ix[2]};
                iy[a] += dir;
                if (in_grid(G, iy) && interior_at(G, phi, iy)) c = CL_GHOST;
            }
    }
    cls[lin] = c;
}

__global__ void k_flag_class(const uint8_t *__restrict__ cls, int64_t nn, uint8_t want, uint8_t want2,
                             uint8_t *__restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    uint8_t c = cls[i];
    flags[i] = (c == want || c == want2) ? 1 : 0;
}

// one thread per 64-node window of an x-row: interior mask
__global__ void k_win_mask(const uint8_t *__restrict__ cls, Geo G, int64_t nwall, int wpr,
                           uint64_t *__restrict__ masks, uint8_t *__restrict__ flags) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwall) return;
    int64_t row = w / wpr;
    int m = (int)(w % wpr);
    int64_t base = row * G.n + (int64_t)m * kWin;
    int cnt = min(kWin, G.n - m * kWin);
    uint64_t mask = 0;
    for (int t = 0; t < cnt; ++t)
        if (cls[base + t] == CL_INTERIOR) mask |= (1ull << t);
    masks[w] = mask;
    flags[w] = mask ? 1 : 0;
}

__global__ void k_make_win(const uint32_t *__restrict__ ids, int64_t nw, const uint64_t *__restrict__ masks,
                           Geo G, int wpr, Win *__restrict__ win) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw) return;
    int64_t w = ids[i];
    int64_t row = w / wpr;
    int m = (int)(w % wpr);
    int j = (G.d > 1) ? (int)(row % G.n) : 0;
    int k = (G.d > 2) ? (int)(row / G.n) : 0;
    Win x;
    x.base = (uint32_t)(row * G.n + (int64_t)m * kWin);
    x.jk = (uint32_t)j | ((uint32_t)k << 16);
    x.mask = masks[w];
    win[i] = x;
}

// ---------------------------------------------------------------- ghosts
__device__ double grad_a(const Geo &G, const double *phi, int64_t lin, const int ix[3], int a) {
    int64_t s = G.st[a];
    if (ix[a] == 0) return __dsub_rn(phi[lin + s], phi[lin]);
    if (ix[a] == G.N) return __dsub_rn(phi[lin], phi[lin - s]);
    return __dmul_rn(0.5, __dsub_rn(phi[lin + s], phi[lin - s]));
}

// multilinear interpolation of grid phi at an index-space point
__device__ double interp_phi(const Geo &G, const double *phi, const double p[3]) {
    int64_t c[3] = {0, 0, 0};
    double t[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < G.d; ++a) {
        double f = floor(p[a]);
        int64_t ci = (int64_t)f;
        if (ci < 0) ci = 0;
        if (ci > G.N - 1) ci = G.N - 1;
        c[a] = ci;
        t[a] = __dsub_rn(p[a], (double)ci);
    }
    double val = 0.0;
    for (int corner = 0; corner < (1 << G.d); ++corner) {
        double w = 1.0;
        int64_t idx = 0;
        for (int a = 0; a < G.d; ++a) {
            int b = (corner >> a) & 1;
            w = __dmul_rn(w, b ? t[a] : __dsub_rn(1.0, t[a]));
            idx += (c[a] + b) * G.st[a];
        }
        val = __dadd_rn(val, __dmul_rn(w, phi[idx]));
    }
    return val;
}

__device__ bool stencil_ok(const Geo &G, const uint8_t *cls, const int ix[3], const int s[3], const int q[3]) {
    int o[3];
    for (o[2] = 0; o[2] <= (G.d > 2 ? q[2] : 0); ++o[2])
        for (o[1] = 0; o[1] <= (G.d > 1 ? q[1] : 0); ++o[1])
            for (o[0] = 0; o[0] <= q[0]; ++o[0]) {
                int iy[3];
                for (int a = 0; a < 3; ++a) iy[a] = ix[a] - (a < G.d ? s[a] * o[a] : 0);
                if (!in_grid(G, iy)) return false;
                if (cls[lin_of(G, iy)] == CL_INACTIVE) return false;
            }
    return true;
}

// Delta tau_OPT(theta): 2 / (G0min + G0max) over the corner frequencies
// A_m (eq. G0minmax_dD); p(A_m) = acosh(1 + m) for m < d and acosh(2d - 1)
// for A_d (eqs. alphaNalpha, alphaNalpha3D).  G0 of Remark exptheta2D (exp)
// or of eqs. G / G3D with coefficients eq. coeff (poly).
__host__ __device__ double dtau_formula(int d, int mode, double cst, double theta) {
    if (mode == BCMG_DTAU_CONST) return cst;
    double gmin = 1e300, gmax = 0.0;
    for (int m = 1; m <= d; ++m) {
        double arg = (m < d) ? (1.0 + m) : (2.0 * d - 1.0);
        double p = acosh(arg);
        double g;
        if (mode == BCMG_DTAU_EXP) {
            g = exp(-p * theta);
        } else {
            double e1 = exp(-p), e2 = exp(-2.0 * p);
            double cm2 = theta * (theta - 1.0) / 2.0;
            double cm1 = theta * (2.0 - theta);
            double c0 = (1.0 - theta) * (2.0 - theta) / 2.0;
            g = cm2 * e2 + cm1 * e1 + c0;
        }
        g = fabs(g);
        gmin = fmin(gmin, g);
        gmax = fmax(gmax, g);
    }
    return 2.0 / (gmin + gmax);
}

struct GhostOut {
    uint16_t *code;
    double *xi, *dt, *eta, *nrm, *Q;
    unsigned long long *nclamp, *nfall;
};

__global__ void k_ghost_setup(const uint32_t *__restrict__ gidx, int64_t ng, const double *__restrict__ phi,
                              const uint8_t *__restrict__ cls, Geo G, int dmode, double dconst, GhostOut out) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int d = G.d;
    int64_t lin = gidx[g];
    int ix[3];
    decode(G, lin, ix);
    // outward normal n = grad phi / |grad phi| (central differences)
    double gr[3] = {0, 0, 0}, n[3] = {0, 0, 0}, key[3] = {0, 0, 0};
    double gn2 = 0.0;
    for (int a = 0; a < d; ++a) {
        gr[a] = grad_a(G, phi, lin, ix, a);
        gn2 = __dadd_rn(gn2, __dmul_rn(gr[a], gr[a]));
    }
    if (gn2 > 0.0) {
        double gnorm = __dsqrt_rn(gn2);
        for (int a = 0; a < d; ++a) {
            n[a] = __ddiv_rn(gr[a], gnorm);
            key[a] = fabs(gr[a]);
        }
    } else {
        bool done = false;
        for (int a = 0; a < d && !done; ++a)
            for (int dir = -1; dir <= 1 && !done; dir += 2) {
                int iy[3] = {ix[0], ix[1], ix[2]};
                iy[a] += dir;
                if (in_grid(G, iy) && cls[lin_of(G, iy)] == CL_INTERIOR) {
                    n[a] = (double)(-dir);
                    done = true;
                }
            }
        for (int a = 0; a < d; ++a) key[a] = fabs(n[a]);
    }
    // eta in [0, 1] with phi(G - eta h n) = 0 by bisection on the
    // multilinear interpolant (64 halvings)
    double eta;
    if (phi[lin] == 0.0) {
        eta = 0.0;
    } else {
        double p1[3];
        for (int a = 0; a < 3; ++a) p1[a] = (a < d) ? __dsub_rn((double)ix[a], n[a]) : (double)ix[a];
        if (interp_phi(G, phi, p1) >= 0.0) {
            eta = 1.0;
            atomicAdd(out.nclamp, 1ull);
        } else {
            double lo = 0.0, hi = 1.0;
            for (int it = 0; it < 64; ++it) {
                double mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
                double pm[3];
                for (int a = 0; a < 3; ++a)
                    pm[a] = (a < d) ? __dsub_rn((double)ix[a], __dmul_rn(mid, n[a])) : (double)ix[a];
                if (interp_phi(G, phi, pm) >= 0.0) lo = mid;
                else hi = mid;
            }
            eta = __dmul_rn(0.5, __dadd_rn(lo, hi));
        }
    }
    // upwind 3^d stencil with G at a corner
    int s[3] = {1, 1, 1}, q[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
        s[a] = (n[a] >= 0.0) ? 1 : -1;
        int far = ix[a] - 2 * s[a];
        if (far < 0 || far > G.N) s[a] = -s[a];
        q[a] = 2;
    }
    if (!stencil_ok(G, cls, ix, s, q)) {
        // axes by increasing |n_a| (stable); per axis: (reversed, 2),
        // (upwind, 1), (reversed, 1), (upwind, 0)
        int order[3] = {0, 1, 2};
        for (int i = 1; i < d; ++i)
            for (int j = i; j > 0 && key[order[j]] < key[order[j - 1]]; --j) {
                int t = order[j];
                order[j] = order[j - 1];
                order[j - 1] = t;
            }
        const int opt_flip[4] = {1, 0, 1, 0};
        const int opt_deg[4] = {2, 1, 1, 0};
        bool ok = false;
        for (int m = 0; m < d && !ok; ++m) {
            int a = order[m];
            int s0 = s[a];
            for (int o = 0; o < 4 && !ok; ++o) {
                int sa = opt_flip[o] ? -s0 : s0;
                int far = ix[a] - sa * opt_deg[o];
                if (far < 0 || far > G.N) continue;
                s[a] = sa;
                q[a] = opt_deg[o];
                ok = stencil_ok(G, cls, ix, s, q);
            }
            if (!ok) {
                s[a] = s0;
                q[a] = 0;
            }
        }
        atomicAdd(out.nfall, 1ull);
    }
    uint16_t code = 0;
    for (int a = 0; a < d; ++a) {
        double xi = __dmul_rn(__dmul_rn((double)s[a], eta), n[a]);
        out.xi[(int64_t)a * ng + g] = xi;
        out.nrm[(int64_t)a * ng + g] = n[a];
        if (s[a] < 0) code |= (uint16_t)(1u << a);
        code |= (uint16_t)((unsigned)q[a] << (3 + 2 * a));
        double xg = __dadd_rn(-1.0, __dmul_rn((double)ix[a], G.h));
        out.Q[g * d + a] = __dsub_rn(xg, __dmul_rn(__dmul_rn(eta, G.h), n[a]));
    }
    out.code[g] = code;
    out.eta[g] = eta;
    out.dt[g] = dtau_formula(d, dmode, dconst, eta);
}

// ---------------------------------------------------------------- band
__global__ void k_band_mark(const uint32_t *__restrict__ gidx, int64_t ng, const uint8_t *__restrict__ cls,
                            Geo G, uint8_t *__restrict__ mark) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    int ix[3];
    decode(G, gidx[g], ix);
    int o[3];
    for (o[2] = (G.d > 2 ? -2 : 0); o[2] <= (G.d > 2 ? 2 : 0); ++o[2])
        for (o[1] = (G.d > 1 ? -2 : 0); o[1] <= (G.d > 1 ? 2 : 0); ++o[1])
            for (o[0] = -2; o[0] <= 2; ++o[0]) {
                int iy[3] = {ix[0] + o[0], ix[1] + o[1], ix[2] + o[2]};
                if (!in_grid(G, iy)) continue;
                int64_t y = lin_of(G, iy);
                if (cls[y] == CL_INACTIVE) mark[y] = 1;
            }
}

__device__ int64_t find_sorted(const uint32_t *a, int64_t n, uint32_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && a[lo] == key) ? lo : -1;
}

__global__ void k_band_setup(const uint32_t *__restrict__ bidx, int64_t nb, const double *__restrict__ phi,
                             const uint8_t *__restrict__ cls, Geo G, int32_t *__restrict__ bref,
                             double *__restrict__ bw) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int64_t lin = bidx[b];
    int ix[3];
    decode(G, lin, ix);
    int32_t ref[3] = {kNoRef, kNoRef, kNoRef};
    double w[3] = {0.0, 0.0, 0.0};
    double den = 0.0;
    for (int a = 0; a < G.d; ++a) {
        double ga = grad_a(G, phi, lin, ix, a);
        if (ga == 0.0) continue;
        int s = ga > 0.0 ? 1 : -1;
        int iy[3] = {ix[0], ix[1], ix[2]};
        iy[a] -= s;
        if (!in_grid(G, iy)) continue;
        int64_t y = lin_of(G, iy);
        if (cls[y] == CL_GHOST) {
            ref[a] = (int32_t)(-y - 1);
        } else {
            int64_t pos = find_sorted(bidx, nb, (uint32_t)y);
            if (pos < 0) continue;
            ref[a] = (int32_t)pos;
        }
        w[a] = fabs(ga);
        den += w[a];
    }
    for (int a = 0; a < 3; ++a) {
        bref[(int64_t)a * nb + b] = ref[a];
        bw[(int64_t)a * nb + b] = (den > 0.0 && ref[a] != kNoRef) ? w[a] / den : 0.0;
    }
}

// ---------------------------------------------------------------- coarsest
__device__ __forceinline__ void lagrange_w(int q, double xi, double w[3]) {
    w[0] = w[1] = w[2] = 0.0;
    if (q == 2) {
        w[0] = (1.0 - xi) * (2.0 - xi) * 0.5;
        w[1] = xi * (2.0 - xi);
        w[2] = xi * (xi - 1.0) * 0.5;
    } else if (q == 1) {
        w[0] = 1.0 - xi;
        w[1] = xi;
    } else {
        w[0] = 1.0;
    }
}

__global__ void k_assemble(const uint32_t *__restrict__ act, int64_t nact, const uint8_t *__restrict__ cls,
                           const uint32_t *__restrict__ gidx, const uint16_t *__restrict__ gcode,
                           const double *__restrict__ gxi, int64_t ng, Geo G, double *__restrict__ A) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nact) return;
    int64_t X = act[r];
    double *row = A + r * nact;
    if (cls[X] == CL_INTERIOR) {
        double ih2 = 1.0 / (G.h * G.h);
        row[r] += 2.0 * G.d * ih2;
        for (int a = 0; a < G.d; ++a)
            for (int dir = -1; dir <= 1; dir += 2) {
                int64_t c = find_sorted(act, nact, (uint32_t)(X + dir * G.st[a]));
                if (c >= 0) row[c] -= ih2;
            }
        return;
    }
    int64_t g = find_sorted(gidx, ng, (uint32_t)X);
    uint16_t code = gcode[g];
    int s[3] = {0, 0, 0}, q[3] = {0, 0, 0};
    double w[3][3] = {{1, 0, 0}, {1, 0, 0}, {1, 0, 0}};
    for (int a = 0; a < G.d; ++a) {
        s[a] = ((code >> a) & 1) ? -1 : 1;
        q[a] = (code >> (3 + 2 * a)) & 3;
        lagrange_w(q[a], gxi[(int64_t)a * ng + g], w[a]);
    }
    for (int o2 = 0; o2 <= q[2]; ++o2)
        for (int o1 = 0; o1 <= q[1]; ++o1)
            for (int o0 = 0; o0 <= q[0]; ++o0) {
                int64_t Y = X - (int64_t)s[0] * o0 * G.st[0] - (int64_t)s[1] * o1 * G.st[1] -
                            (int64_t)s[2] * o2 * G.st[2];
                int64_t c = find_sorted(act, nact, (uint32_t)Y);
                if (c >= 0) row[c] += w[0][o0] * w[1][o1] * w[2][o2];
            }
}

__global__ void k_identity(double *__restrict__ M, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * n) return;
    M[i] = (i / n == i % n) ? 1.0 : 0.0;
}

// Gauss-Jordan step k, part 1 (one block): partial pivoting, row swap,
// scaling of the pivot row, and the column of elimination factors.
__global__ void k_gj_pivot(double *__restrict__ A, double *__restrict__ B, int64_t n, int64_t k,
                           double *__restrict__ col, int *__restrict__ singular) {
    __shared__ double bv[1024];
    __shared__ int64_t bi[1024];
    __shared__ double piv;
    double best = -1.0;
    int64_t bidx = n;
    for (int64_t i = k + threadIdx.x; i < n; i += blockDim.x) {
        double v = fabs(A[i * n + k]);
        if (v > best || (v == best && i < bidx)) {
            best = v;
            bidx = i;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bidx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double v = bv[threadIdx.x + s];
            int64_t ii = bi[threadIdx.x + s];
            if (v > bv[threadIdx.x] || (v == bv[threadIdx.x] && ii < bi[threadIdx.x])) {
                bv[threadIdx.x] = v;
                bi[threadIdx.x] = ii;
            }
        }
        __syncthreads();
    }
    int64_t p = bi[0];
    if (bv[0] <= 0.0) {
        if (threadIdx.x == 0) *singular = 1;
        p = k;
    }
    if (p != k)
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            double t = A[k * n + j];
            A[k * n + j] = A[p * n + j];
            A[p * n + j] = t;
            t = B[k * n + j];
            B[k * n + j] = B[p * n + j];
            B[p * n + j] = t;
        }
    __syncthreads();
    if (threadIdx.x == 0) piv = A[k * n + k];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) col[i] = (i == k) ? 0.0 : A[i * n + k];
    __syncthreads();
    double ip = (piv != 0.0) ? 1.0 / piv : 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        A[k * n + j] *= ip;
        B[k * n + j] *= ip;
    }
}

// Gauss-Jordan step k, part 2: eliminate column k from every other row.
__global__ void k_gj_elim(double *__restrict__ A, double *__restrict__ B, int64_t n, int64_t k,
                          const double *__restrict__ col) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * n) return;
    int64_t i = t / n, j = t % n;
    if (i == k) return;
    double f = col[i];
    if (f == 0.0) return;
    A[i * n + j] -= f * A[k * n + j];
    B[i * n + j] -= f * B[k * n + j];
}

inline int nblocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

double dtau_of(int d, int mode, double cst, double theta) { return dtau_formula(d, mode, cst, theta); }

int64_t compact_flags(Handle &H, const uint8_t *flags, int64_t n, uint32_t **out, bool temp) {
    int64_t nblk = (n + kCompactTile - 1) / kCompactTile;
    if (nblk == 0) nblk = 1;
    int64_t *counts = (int64_t *)dalloc(H, sizeof(int64_t) * nblk, true);
    k_count<<<(unsigned)nblk, kCompactThreads, 0, H.st>>>(flags, n, counts);
    count_launch(H);
    check_cuda(cudaGetLastError(), "k_count");
    std::vector<int64_t> hc(nblk);
    check_cuda(cudaMemcpyAsync(hc.data(), counts, sizeof(int64_t) * nblk, cudaMemcpyDeviceToHost, H.st),
               "compact counts");
    check_cuda(cudaStreamSynchronize(H.st), "compact sync");
    int64_t total = 0;
    for (int64_t i = 0; i < nblk; ++i) {
        int64_t c = hc[i];
        hc[i] = total;
        total += c;
    }
    check_cuda(cudaMemcpyAsync(counts, hc.data(), sizeof(int64_t) * nblk, cudaMemcpyHostToDevice, H.st),
               "compact offsets");
    *out = (uint32_t *)dalloc(H, sizeof(uint32_t) * (size_t)std::max<int64_t>(total, 1), temp);
    k_scatter<<<(unsigned)nblk, kCompactThreads, 0, H.st>>>(flags, n, counts, *out);
    count_launch(H);
    check_cuda(cudaGetLastError(), "k_scatter");
    check_cuda(cudaStreamSynchronize(H.st), "compact sync 2");
    return total;
}

void setup_level(Handle &H, Level &L, int li) {
    Geo G = geo_of(L);
    const int T = 256;
    // phi of this level by injection from the finer level
    if (li > 0) {
        Level &Lf = H.L[li - 1];
        double *phic = (double *)dalloc(H, sizeof(double) * L.nn, true);
        k_inject<<<nblocks(L.nn, T), T, 0, H.st>>>(Lf.phi, geo_of(Lf), G, phic);
        count_launch(H);
        check_cuda(cudaGetLastError(), "k_inject");
        L.phi = phic;
    }
    L.cls = (uint8_t *)dalloc(H, L.nn);
    k_classify<<<nblocks(L.nn, T), T, 0, H.st>>>(L.phi, G, L.nn, L.cls);
    count_launch(H);
    check_cuda(cudaGetLastError(), "k_classify");

    uint8_t *flags = (uint8_t *)dalloc(H, (size_t)L.nn + 1, true);
    // interior windows
    int wpr = (L.n + kWin - 1) / kWin;
    int64_t rows = L.nn / L.n;
    int64_t nwall = rows * wpr;
    uint64_t *masks = (uint64_t *)dalloc(H, sizeof(uint64_t) * nwall, true);
    k_win_mask<<<nblocks(nwall, T), T, 0, H.st>>>(L.cls, G, nwall, wpr, masks, flags);
    count_launch(H);
    check_cuda(cudaGetLastError(), "k_win_mask");
    uint32_t *ids = nullptr;
    L.nwin = compact_flags(H, flags, nwall, &ids, true);
    L.win = (Win *)dalloc(H, sizeof(Win) * (size_t)std::max<int64_t>(L.nwin, 1));
    if (L.nwin > 0) {
        k_make_win<<<nblocks(L.nwin, T), T, 0, H.st>>>(ids, L.nwin, masks, G, wpr, L.win);
        count_launch(H);
        check_cuda(cudaGetLastError(), "k_make_win");
    }
    // counts of interior / boxdir nodes
    k_flag_class<<<nblocks(L.nn, T), T, 0, H.st>>>(L.cls, L.nn, CL_INTERIOR, CL_INTERIOR, flags);
    count_launch(H);
    uint32_t *tmpidx = nullptr;
    L.nint = compact_flags(H, flags, L.nn, &tmpidx, true);
    k_flag_class<<<nblocks(L.nn, T), T, 0, H.st>>>(L.cls, L.nn, CL_BOXDIR, CL_BOXDIR, flags);
    count_launch(H);
    L.nbox = compact_flags(H, flags, L.nn, &L.boxidx);
    if (L.nint == 0) return;

    // ghost list and per-ghost geometry
    k_flag_class<<<nblocks(L.nn, T), T, 0, H.st>>>(L.cls, L.nn, CL_GHOST, CL_GHOST, flags);
    count_launch(H);
    L.ng = compact_flags(H, flags, L.nn, &L.gidx);
    int64_t ng1 = std::max<int64_t>(L.ng, 1);
    L.gcode = (uint16_t *)dalloc(H, sizeof(uint16_t) * ng1);
    L.gxi = (double *)dalloc(H, sizeof(double) * 3 * ng1);
    L.gn = (double *)dalloc(H, sizeof(double) * 3 * ng1);
    L.gdt = (double *)dalloc(H, sizeof(double) * ng1);
    L.geta = (double *)dalloc(H, sizeof(double) * ng1);
    L.gQ = (double *)dalloc(H, sizeof(double) * 3 * ng1);
    L.gtmp = (double *)dalloc(H, sizeof(double) * ng1);
    unsigned long long *cnt = (unsigned long long *)dalloc(H, 2 * sizeof(unsigned long long), true);
    if (L.ng > 0) {
        GhostOut go{L.gcode, L.gxi, L.gdt, L.geta, L.gn, L.gQ, cnt, cnt + 1};
        k_ghost_setup<<<nblocks(L.ng, 128), 128, 0, H.st>>>(L.gidx, L.ng, L.phi, L.cls, G, H.o.dtau_mode,
                                                            H.o.dtau_const, go);
        count_launch(H);
        check_cuda(cudaGetLastError(), "k_ghost_setup");
    }
    unsigned long long hcnt[2] = {0, 0};
    check_cuda(cudaMemcpyAsync(hcnt, cnt, sizeof(hcnt), cudaMemcpyDeviceToHost, H.st), "ghost counts");
    // band: inactive nodes within Chebyshev distance 2 of a ghost
    check_cuda(cudaMemsetAsync(flags, 0, (size_t)L.nn, H.st), "band memset");
    if (L.ng > 0) {
        k_band_mark<<<nblocks(L.ng, T), T, 0, H.st>>>(L.gidx, L.ng, L.cls, G, flags);
        count_launch(H);
        check_cuda(cudaGetLastError(), "k_band_mark");
    }
    L.nb = compact_flags(H, flags, L.nn, &L.bidx);
    L.nclamp = (int64_t)hcnt[0];
    L.nfall = (int64_t)hcnt[1];
    int64_t nb1 = std::max<int64_t>(L.nb, 1);
    L.bref = (int32_t *)dalloc(H, sizeof(int32_t) * 3 * nb1);
    L.bw = (double *)dalloc(H, sizeof(double) * 3 * nb1);
    L.bbuf = (double *)dalloc(H, sizeof(double) * 2 * nb1);
    if (L.nb > 0) {
        k_band_setup<<<nblocks(L.nb, T), T, 0, H.st>>>(L.bidx, L.nb, L.phi, L.cls, G, L.bref, L.bw);
        count_launch(H);
        check_cuda(cudaGetLastError(), "k_band_setup");
    }
    // level arrays
    if (li > 0) L.u = (double *)dalloc(H, sizeof(double) * L.nn);
    L.F = (double *)dalloc(H, sizeof(double) * L.nn);
    L.r = (double *)dalloc(H, sizeof(double) * L.nn);
    check_cuda(cudaStreamSynchronize(H.st), "setup_level sync");
}

void setup_coarsest(Handle &H, Level &L) {
    Geo G = geo_of(L);
    const int T = 256;
    uint8_t *flags = (uint8_t *)dalloc(H, (size_t)L.nn + 1, true);
    k_flag_class<<<nblocks(L.nn, T), T, 0, H.st>>>(L.cls, L.nn, CL_INTERIOR, CL_GHOST, flags);
    count_launch(H);
    L.nact = compact_flags(H, flags, L.nn, &L.act);
    if (L.nact > kMaxCoarse) throw Error{BCMG_EGEOM, "coarsest system has more than 4096 unknowns"};
    int64_t n = L.nact;
    double *A = (double *)dalloc(H, sizeof(double) * std::max<int64_t>(n * n, 1), true);
    L.Ainv = (double *)dalloc(H, sizeof(double) * std::max<int64_t>(n * n, 1));
    L.crhs = (double *)dalloc(H, sizeof(double) * std::max<int64_t>(n, 1));
    double *col = (double *)dalloc(H, sizeof(double) * std::max<int64_t>(n, 1), true);
    int *sing = (int *)dalloc(H, sizeof(int), true);
    k_assemble<<<nblocks(n, 128), 128, 0, H.st>>>(L.act, n, L.cls, L.gidx, L.gcode, L.gxi, L.ng, G, A);
    count_launch(H);
    check_cuda(cudaGetLastError(), "k_assemble");
    k_identity<<<nblocks(n * n, T), T, 0, H.st>>>(L.Ainv, n);
    count_launch(H);
    for (int64_t k = 0; k < n; ++k) {
        k_gj_pivot<<<1, 1024, 0, H.st>>>(A, L.Ainv, n, k, col, sing);
        count_launch(H);
        k_gj_elim<<<nblocks(n * n, T), T, 0, H.st>>>(A, L.Ainv, n, k, col);
        count_launch(H);
    }
    check_cuda(cudaGetLastError(), "gauss-jordan");
    int hs = 0;
    check_cuda(cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, H.st), "singular flag");
    check_cuda(cudaStreamSynchronize(H.st), "coarsest sync");
    if (hs) throw Error{BCMG_EGEOM, "coarsest system is singular"};
}

}  // namespace bcmg
