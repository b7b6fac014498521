// Hierarchy set-up on the GPU: per-level node classes, interior lists,
// ghost projection / stencil / Delta tau, band lists and the coarsest-level
// inverse (arXiv 2207.14208, Sec. 3.3 geometry, Sec. 3.2-4.1 BLFA).
//
// The geometric decisions (classes, normals, the bisection for eta, the
// stencil directions and fall-backs, band membership) use explicitly rounded
// IEEE operations so that they do not depend on FMA contraction.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <set>

#include "bcmg_internal.cuh"

namespace bcmg {

namespace {

struct Geo {
    int d, N, n;
    int64_t st[3];
    double h, lo;
};

Geo geo_of(const Level &L) {
    Geo g;
    g.d = L.d;
    g.N = L.N;
    g.n = L.n;
    for (int a = 0; a < 3; ++a) g.st[a] = L.st[a];
    g.h = L.h;
    g.lo = L.lo;
    return g;
}

// node indices are below 2^32 (checked at creation): 32-bit division
__device__ __forceinline__ void decode(const Geo &G, int64_t lin, int ix[3]) {
    uint32_t v = (uint32_t)lin;
    const uint32_t n = (uint32_t)G.n;
    ix[0] = ix[1] = ix[2] = 0;
    for (int a = 0; a < G.d; ++a) {
        const uint32_t q = v / n;
        ix[a] = (int)(v - q * n);
        v = q;
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

// Compaction of up to four lists from one byte array in one pass each: list
// b holds, in increasing order, the indices i with flags[i] & mask_b != 0
// (masks packed one per byte in `masks`).  Per block: the count of each
// list (counts[base + block * nl + b]); then the scatter, whose per-thread
// counts (at most kCompactPerThread each) are scanned as four 16-bit fields
// of one 64-bit word (a block holds at most 4096 items, so no field
// overflows).  Every flag array of a set-up round goes in one launch: the
// blocks of array k start at blk0[k].
constexpr int kCompactMax = 24;  // flag arrays per launch

struct CompactArr {
    const uint8_t *flags;
    int64_t n;
    int64_t blk0;   // first block of this array
    int64_t base;   // its first count slot
    uint32_t masks;
    int nl;
    uint32_t *out[4];  // nullptr: list counted only
};

struct CompactBatch {
    int narr;
    CompactArr a[kCompactMax];
};

__device__ __forceinline__ int compact_arr_of(const CompactBatch &B) {
    int k = 0;
    for (int i = 1; i < B.narr; ++i)
        if ((int64_t)blockIdx.x >= B.a[i].blk0) k = i;
    return k;
}

// this thread's kCompactPerThread flag bytes as four little-endian words
// (one 16-byte load when the whole run is in range and aligned; zero past
// the end)
__device__ __forceinline__ void compact_load(const CompactArr &A, int64_t base, uint32_t w[4]) {
    const bool vec = base + kCompactPerThread <= A.n && ((reinterpret_cast<uintptr_t>(A.flags + base) & 15) == 0);
    if (vec) {
        const uint4 v = *reinterpret_cast<const uint4 *>(A.flags + base);
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t x = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t i = base + 4 * q + r;
                x |= (uint32_t)(i < A.n ? A.flags[i] : (uint8_t)0) << (8 * r);
            }
            w[q] = x;
        }
    }
}

// bit i of the result: byte i of the 16 has a bit of mask m (byte-parallel:
// the high bit of each byte of ((t & 0x7f..) + 0x7f..) | t is set iff the
// byte of t is non-zero)
__device__ __forceinline__ uint32_t compact_hitmask(const uint32_t w[4], uint32_t m) {
    const uint32_t mm = m * 0x01010101u;
    uint32_t hm = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t t = w[q] & mm;
        const uint32_t nz = (((t & 0x7f7f7f7fu) + 0x7f7f7f7fu) | t) & 0x80808080u;
        hm |= (((nz >> 7) & 1u) | ((nz >> 14) & 2u) | ((nz >> 21) & 4u) | ((nz >> 28) & 8u)) << (4 * q);
    }
    return hm;
}

// the counts of the (up to four) lists as 16-bit fields
__device__ __forceinline__ uint64_t compact_hits(const uint32_t w[4], uint32_t masks, int nl) {
    uint64_t c = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if (b < nl) c += (uint64_t)__popc(compact_hitmask(w, (masks >> (8 * b)) & 0xffu)) << (16 * b);
    return c;
}

__global__ void __launch_bounds__(kCompactThreads) k_count(CompactBatch B, int64_t *__restrict__ counts) {
    __shared__ uint64_t red[kCompactThreads / 32];
    const CompactArr &A = B.a[compact_arr_of(B)];
    const int64_t blk = (int64_t)blockIdx.x - A.blk0;
    const int64_t base = blk * kCompactTile + (int64_t)threadIdx.x * kCompactPerThread;
    uint32_t w[4];
    compact_load(A, base, w);
    uint64_t c = compact_hits(w, A.masks, A.nl);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) red[warp] = c;
    __syncthreads();
    if (threadIdx.x < A.nl) {
        uint64_t t = 0;
        for (int w = 0; w < kCompactThreads / 32; ++w) t += red[w];
        counts[A.base + blk * A.nl + threadIdx.x] = (int64_t)((t >> (16 * threadIdx.x)) & 0xffffu);
    }
}

__global__ void __launch_bounds__(kCompactThreads) k_scatter(CompactBatch B, const int64_t *__restrict__ offs) {
    __shared__ uint64_t sc[kCompactThreads / 32];
    const CompactArr &A = B.a[compact_arr_of(B)];
    if (!A.out[0] && !A.out[1] && !A.out[2] && !A.out[3]) return;  // counted only (uniform per block)
    const int64_t blk = (int64_t)blockIdx.x - A.blk0;
    const int64_t base = blk * kCompactTile + (int64_t)threadIdx.x * kCompactPerThread;
    uint32_t w[4];
    compact_load(A, base, w);
    const uint64_t c = compact_hits(w, A.masks, A.nl);
    // exclusive scan over the block: warp scans, then a scan of the warp
    // totals by warp 0 (integer, deterministic)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sc[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < kCompactThreads / 32 ? sc[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kCompactThreads / 32) sc[lane] = w;
    }
    __syncthreads();
    const uint64_t excl = x - c + (warp > 0 ? sc[warp - 1] : 0);
    // each list's hits in increasing index order from the thread's offset
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        if (b >= A.nl || !A.out[b]) continue;
        int64_t pos = offs[A.base + blk * A.nl + b] + (int64_t)((excl >> (16 * b)) & 0xffffu);
        uint32_t hm = compact_hitmask(w, (A.masks >> (8 * b)) & 0xffu);
        while (hm) {
            A.out[b][pos++] = (uint32_t)(base + __ffs(hm) - 1);
            hm &= hm - 1;
        }
    }
}

// ---------------------------------------------------------------- classes
// x < 0.0 decided on the IEEE bit pattern (sign set, not -0, not NaN), so
// the test runs on the integer pipe instead of the FP64 pipe
__device__ __forceinline__ bool neg_d(double x) {
    const long long b = __double_as_longlong(x);
    const long long m = b & 0x7fffffffffffffffLL;
    return b < 0 && m != 0 && m <= 0x7ff0000000000000LL;
}

// Node classes of one level (Sec. 3.3) and, packed in one byte per node, the
// flags of every list the set-up compacts (red / black interior, box-edge
// Dirichlet, ghost, active), one thread per node on a (x-blocks, j, k) grid
// (no index division).
// list flags of a node; a black interior node with a neighbour that is not
// interior (a ghost or a box-edge node) is also listed apart (kFlBNear), so
// that the cycle's residual after a smoothing step finds the black rows
// whose residual the ghost relaxation may have changed
enum : uint8_t { kFlRed = 1, kFlBlack = 2, kFlBox = 4, kFlGhost = 8, kFlAct = 16, kFlBNear = 32 };

// One launch classifies every candidate level.  Level l reads the finest
// phi at stride 2^l (the injection, Sec. 2.1) and, for l > 0, stores its
// phi.  Threads of a 32 x 4 block own (i, j) columns and march a chunk of
// kClassPlanes planes in k, keeping phi of planes k - 1, k, k + 1 in
// registers, so each phi value is read from memory about once per column
// step besides the four in-plane neighbours (which the block's other threads
// read too: cache hits).
constexpr int kClassPlanes = 8;
constexpr int kClassMax = 24;

struct ClassLevel {
    Geo G;
    int s;                 // stride in the finest grid (2^l)
    double *phic;          // this level's phi (nullptr on the finest)
    uint8_t *cls, *flags;
    int64_t blk0;          // first block
    int bx, by;            // blocks along i and j (chunks along k follow)
};

struct ClassBatch {
    int nl;
    const double *phi0;
    int64_t st0[3];        // strides of the finest grid
    ClassLevel lv[kClassMax];
};

template <int D>
__global__ void __launch_bounds__(128) k_classify(ClassBatch B) {
    int l = 0;
    for (int q = 1; q < B.nl; ++q)
        if ((int64_t)blockIdx.x >= B.lv[q].blk0) l = q;
    const ClassLevel &C = B.lv[l];
    const int N = C.G.N;
    // node indices fit 32 bits (checked at creation), so does the block count
    const uint32_t bl = (uint32_t)((int64_t)blockIdx.x - C.blk0);
    const uint32_t bxy = (uint32_t)C.bx * (uint32_t)C.by;
    const uint32_t ch = bl / bxy, r = bl - ch * bxy, byi = r / (uint32_t)C.bx, bxi = r - byi * (uint32_t)C.bx;
    const int i = (int)bxi * 32 + threadIdx.x, j = (int)byi * 4 + threadIdx.y;
    if (i > N || j > N) return;
    const int k0 = (D == 3) ? (int)ch * kClassPlanes : 0;
    const int nk = (D == 3) ? min(kClassPlanes, N + 1 - k0) : 1;
    const uint32_t s0 = (uint32_t)C.s, s1 = (uint32_t)C.s * (uint32_t)B.st0[1];
    const uint32_t s2 = (D == 3) ? (uint32_t)C.s * (uint32_t)B.st0[2] : 0u;
    const uint32_t sy = (uint32_t)C.G.st[1], sz = (D == 3) ? (uint32_t)C.G.st[2] : 0u;
    // a neighbour counts when it is off the box edge (all coordinates
    // strictly inside) and has phi < 0; the in-plane part of that test is
    // fixed per column
    const bool inx = j > 0 && j < N, iny = i > 0 && i < N;
    const bool xm = (i - 1 > 0) && inx, xp = (i + 1 < N) && inx;
    const bool ym = (j - 1 > 0) && iny, yp = (j + 1 < N) && iny;
    const bool zin = inx && iny;
    const bool edge_ij = i == 0 || i == N || j == 0 || j == N;
    const uint8_t par0 = (uint8_t)((i + j + k0) & 1);
    const double *p = B.phi0 + ((uint32_t)i * s0 + (uint32_t)j * s1 + (uint32_t)k0 * s2);
    uint32_t lin = (uint32_t)i + (uint32_t)j * sy + (uint32_t)k0 * sz;
    // the column's phi on planes k0 - 1 .. k0 + kClassPlanes, all loads in
    // flight together
    constexpr int NP = (D == 3) ? kClassPlanes + 2 : 3;
    double pz[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int kk = k0 - 1 + q;
        pz[q] = (D == 3) ? ((kk >= 0 && kk <= N) ? p[(int)(q - 1) * (int64_t)s2] : 0.0) : (q == 1 ? p[0] : 0.0);
    }
#pragma unroll
    for (int q = 0; q < NP - 2; ++q) {
        if (q >= nk) break;
        const int k = k0 + q;
        const double pc = pz[q + 1];
        if (C.phic) C.phic[lin] = pc;
        // the four in-plane neighbours are loaded together (predicated on
        // the box, not branched on one another)
        const bool inz = (D == 2) || (k > 0 && k < N);
        const double ax = (inz && xm) ? p[-(int64_t)s0] : 1.0, bx = (inz && xp) ? p[s0] : 1.0;
        const double ay = (inz && ym) ? p[-(int64_t)s1] : 1.0, by = (inz && yp) ? p[s1] : 1.0;
        bool gh = neg_d(ax) | neg_d(bx) | neg_d(ay) | neg_d(by);
        if (D == 3) gh = gh | (zin & (k - 1 > 0) & neg_d(pz[q])) | (zin & (k + 1 < N) & neg_d(pz[q + 2]));
        const bool edge = edge_ij || (D == 3 && (k == 0 || k == N));
        const uint8_t c = neg_d(pc) ? (edge ? CL_BOXDIR : CL_INTERIOR) : (gh ? CL_GHOST : CL_INACTIVE);
        C.cls[lin] = c;
        uint8_t fl = 0;
        if (c == CL_INTERIOR && (par0 ^ (uint8_t)(q & 1)) != 0) {
            // black: listed apart unless every neighbour is interior (off the
            // box edge with phi < 0: the test above, whose edge neighbours
            // read as phi = 1), i.e. when a ghost or a box-edge node is next
            // to it
            bool all_int = neg_d(ax) & neg_d(bx) & neg_d(ay) & neg_d(by);
            if (D == 3) all_int = all_int & (k - 1 > 0) & neg_d(pz[q]) & (k + 1 < N) & neg_d(pz[q + 2]);
            fl = kFlBlack | (all_int ? 0 : kFlBNear) | kFlAct;
        } else if (c == CL_INTERIOR) fl = kFlRed | kFlAct;
        else if (c == CL_GHOST) fl = kFlGhost | kFlAct;
        else if (c == CL_BOXDIR) fl = kFlBox;
        C.flags[lin] = fl;
        p += s2;
        lin += sz;
    }
}

// bit j of bits: black entry j (blist[j]) has the kFlBNear flag; a warp
// writes one word (every thread reaches the ballot).  Every level in one
// launch: the blocks of level q start at blk0[q].
constexpr int kNearMax = 32;  // levels of one launch
struct NearLevel {
    const uint32_t *blist;
    const uint8_t *flags;
    uint32_t *bits;
    int64_t nb, blk0;
};
struct NearBatch {
    int nl;
    NearLevel lv[kNearMax];
};

__global__ void __launch_bounds__(256) k_near_bits(NearBatch B) {
    int q = 0;
    for (int k = 1; k < B.nl; ++k)
        if ((int64_t)blockIdx.x >= B.lv[k].blk0) q = k;
    const NearLevel &L = B.lv[q];
    const int64_t j = ((int64_t)blockIdx.x - L.blk0) * blockDim.x + threadIdx.x;
    const bool near = j < L.nb && (L.flags[L.blist[j]] & kFlBNear) != 0;
    const unsigned w = __ballot_sync(0xffffffffu, near);
    if ((threadIdx.x & 31) == 0 && j < L.nb) L.bits[j >> 5] = w;
}

// ---------------------------------------------------------------- ghosts
__device__ double grad_a(const Geo &G, const double *phi, int64_t lin, const int ix[3], int a) {
    int64_t s = G.st[a];
    if (ix[a] == 0) return __dsub_rn(phi[lin + s], phi[lin]);
    if (ix[a] == G.N) return __dsub_rn(phi[lin], phi[lin - s]);
    return __dmul_rn(0.5, __dsub_rn(phi[lin + s], phi[lin - s]));
}

// multilinear interpolation of grid phi at an index-space point.  The corner
// values of the last cell are kept in registers (every point of one ghost's
// bisection lies in the same cell or two), so the serial bisection chain
// does not wait on global loads.
struct CellCache {
    int64_t c[3] = {-1, -1, -1};
    double v[8];
};

__device__ __forceinline__ double interp_phi(const Geo &G, const double *phi, const double p[3], CellCache &cc) {
    int64_t c[3] = {0, 0, 0};
    double t[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= G.d) break;
        double f = floor(p[a]);
        int64_t ci = (int64_t)f;
        if (ci < 0) ci = 0;
        if (ci > G.N - 1) ci = G.N - 1;
        c[a] = ci;
        t[a] = __dsub_rn(p[a], (double)ci);
    }
    if (c[0] != cc.c[0] || c[1] != cc.c[1] || c[2] != cc.c[2]) {
#pragma unroll
        for (int corner = 0; corner < 8; ++corner) {
            if (corner >= (1 << G.d)) break;
            int64_t idx = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (a < G.d) idx += (c[a] + ((corner >> a) & 1)) * G.st[a];
            cc.v[corner] = phi[idx];
        }
        cc.c[0] = c[0];
        cc.c[1] = c[1];
        cc.c[2] = c[2];
    }
    // corner weights prod_a (b_a ? t_a : 1 - t_a), multiplied in axis order
    // (the leading 1.0 factor is exact and dropped), the x-y products shared
    // by the corners that differ only in z; sum in corner order
    double f[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f[a][0] = (a < G.d) ? __dsub_rn(1.0, t[a]) : 1.0;
        f[a][1] = t[a];
    }
    double p01[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) p01[k] = (G.d >= 2) ? __dmul_rn(f[0][k & 1], f[1][k >> 1]) : f[0][k & 1];
    double val = 0.0;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        if (corner >= (1 << G.d)) break;
        const double w = (G.d == 3) ? __dmul_rn(p01[corner & 3], f[2][corner >> 2]) : p01[corner & 3];
        val = __dadd_rn(val, __dmul_rn(w, cc.v[corner]));
    }
    return val;
}

__device__ __forceinline__ bool stencil_ok(const Geo &G, const uint8_t *cls, const int ix[3], const int s[3], const int q[3]) {
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
// for A_d (eqs. alphaNalpha, alphaNalpha3D).  Dirichlet: G0 of Remark
// exptheta2D, exp(-p theta) (exp), or of eqs. G / G3D with coefficients
// eq. coeff (poly).  Neumann: p exp(-p theta) (Remark exptheta2D) or eq. GN
// with coefficients eq. coeffN; the result is Delta tau / h (eqs.
// dtauoptLFA_Neumann, dtauoptLFA3D_Neumann).
// The corner exponents p(A_m), m = 1..d, depend on d only: computed once on
// the host and passed to every ghost.
struct DtauP {
    double p[3];
};

DtauP dtau_p(int d) {
    DtauP r{};
    for (int m = 1; m <= d && m <= 3; ++m) r.p[m - 1] = acosh((m < d) ? (1.0 + m) : (2.0 * d - 1.0));
    return r;
}

__host__ __device__ double dtau_formula(int d, int bc, int mode, double cst, double theta, const DtauP &P) {
    if (mode == BCMG_DTAU_CONST) return cst;
    double gmin = 1e300, gmax = 0.0;
    for (int m = 1; m <= d; ++m) {
        const double p = P.p[m - 1];
        double g;
        if (mode == BCMG_DTAU_EXP) {
            g = (bc == BCMG_BC_NEUMANN) ? p * exp(-p * theta) : exp(-p * theta);
        } else {
            double e1 = exp(-p), e2 = exp(-2.0 * p);
            double cm2, cm1, c0;
            if (bc == BCMG_BC_NEUMANN) {
                cm2 = 0.5 - theta;
                cm1 = 2.0 * (theta - 1.0);
                c0 = 1.5 - theta;
            } else {
                cm2 = theta * (theta - 1.0) / 2.0;
                cm1 = theta * (2.0 - theta);
                c0 = (1.0 - theta) * (2.0 - theta) / 2.0;
            }
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

// geometry of ghost g of one level (normal, eta, stencil, xi, Q, Delta tau);
// the dimension is a template argument so that the per-axis arrays stay in
// registers
template <int D>
__device__ __forceinline__ void ghost_one(int bc, const uint32_t *__restrict__ gidx, int64_t ng, const double *__restrict__ phi,
                          const uint8_t *__restrict__ cls, const Geo &G, int dmode, double dconst, const DtauP &P,
                          const GhostOut &out, int64_t g) {
    constexpr int d = D;
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
    CellCache cc;
    if (phi[lin] == 0.0) {
        eta = 0.0;
    } else {
        double p1[3];
        for (int a = 0; a < 3; ++a) p1[a] = (a < d) ? __dsub_rn((double)ix[a], n[a]) : (double)ix[a];
        if (interp_phi(G, phi, p1, cc) >= 0.0) {
            eta = 1.0;
            atomicAdd(out.nclamp, 1ull);
        } else {
            // For eta in (0, 1) the point G - eta h n stays in one grid cell
            // (|n_a| <= 1), the one holding G - h n / 2, where the
            // multilinear interpolant is a polynomial of degree d in eta:
            // t_a(eta) = (i_a - c_a) - n_a eta.  Its coefficients are built
            // once (x, then y, then z) and the halving runs on them (Horner);
            // eta then differs from a pointwise evaluation only in rounding.
            int c[3] = {0, 0, 0};
            double al[3] = {0.0, 0.0, 0.0}, be[3] = {0.0, 0.0, 0.0};
            for (int a = 0; a < d; ++a) {
                const double pmid = __dsub_rn((double)ix[a], __dmul_rn(0.5, n[a]));
                int ci = (int)floor(pmid);
                ci = max(0, min(G.N - 1, ci));
                c[a] = ci;
                al[a] = (double)(ix[a] - ci);
                be[a] = -n[a];
            }
            double v[8];
            for (int k = 0; k < (1 << d); ++k) {
                int64_t idx = 0;
                for (int a = 0; a < d; ++a) idx += (int64_t)(c[a] + ((k >> a) & 1)) * G.st[a];
                v[k] = phi[idx];
            }
            // factors (1 - t_a) and t_a as (constant, slope) pairs
            double f0[3][2], f1[3][2];
            for (int a = 0; a < d; ++a) {
                f1[a][0] = al[a];
                f1[a][1] = be[a];
                f0[a][0] = 1.0 - al[a];
                f0[a][1] = -be[a];
            }
            // along x: 2^(d-1) linear polynomials
            double gx[4][2];
            for (int k = 0; k < (1 << (d - 1)); ++k) {
                const double v0 = v[2 * k], v1 = v[2 * k + 1];
                gx[k][0] = v0 * f0[0][0] + v1 * f1[0][0];
                gx[k][1] = v0 * f0[0][1] + v1 * f1[0][1];
            }
            // along y: 2^(d-2) quadratics
            double gy[2][3];
            for (int k = 0; k < (1 << (d - 2)); ++k) {
                const double *a0 = gx[2 * k], *a1 = gx[2 * k + 1];
                gy[k][0] = a0[0] * f0[1][0] + a1[0] * f1[1][0];
                gy[k][1] = a0[0] * f0[1][1] + a0[1] * f0[1][0] + a1[0] * f1[1][1] + a1[1] * f1[1][0];
                gy[k][2] = a0[1] * f0[1][1] + a1[1] * f1[1][1];
            }
            double cf[4] = {gy[0][0], gy[0][1], gy[0][2], 0.0};
            if (d == 3) {  // along z: the cubic
                const double *a0 = gy[0], *a1 = gy[1];
                cf[0] = a0[0] * f0[2][0] + a1[0] * f1[2][0];
                cf[1] = a0[0] * f0[2][1] + a0[1] * f0[2][0] + a1[0] * f1[2][1] + a1[1] * f1[2][0];
                cf[2] = a0[1] * f0[2][1] + a0[2] * f0[2][0] + a1[1] * f1[2][1] + a1[2] * f1[2][0];
                cf[3] = a0[2] * f0[2][1] + a1[2] * f1[2][1];
            }
            // once the midpoint rounds onto an end of the interval, every
            // remaining halving leaves eta = that midpoint: stop there.
            // lo, hi and mid lie in [0, 1] with lo + hi >= 2^-64, so the
            // halving is an exponent decrement and the comparisons are on
            // bit patterns (equal doubles have equal bits here; val >= 0
            // is "sign bit clear, or -0"), keeping them off the FP64 pipe
            const long long kHalf = 1LL << 52, kSign = (long long)0x8000000000000000ULL;
            double lo = 0.0, hi = 1.0;
            for (int it = 0; it < 64; ++it) {
                const double mid = __longlong_as_double(__double_as_longlong(__dadd_rn(lo, hi)) - kHalf);
                const long long bm = __double_as_longlong(mid);
                if (bm == __double_as_longlong(lo) || bm == __double_as_longlong(hi)) {
                    lo = hi = mid;
                    break;
                }
                const long long bv = __double_as_longlong(fma(fma(fma(cf[3], mid, cf[2]), mid, cf[1]), mid, cf[0]));
                if (bv >= 0 || bv == kSign) lo = mid;
                else hi = mid;
            }
            eta = __longlong_as_double(__double_as_longlong(__dadd_rn(lo, hi)) - kHalf);
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
        double xg = __dadd_rn(G.lo, __dmul_rn((double)ix[a], G.h));
        out.Q[g * d + a] = __dsub_rn(xg, __dmul_rn(__dmul_rn(eta, G.h), n[a]));
    }
    out.code[g] = code;
    out.eta[g] = eta;
    // Neumann: the formula gives Delta tau / h
    out.dt[g] = dtau_formula(d, bc, dmode, dconst, eta, P) * (bc == BCMG_BC_NEUMANN ? G.h : 1.0);
}

// ---------------------------------------------------------------- band
// mark the inactive nodes within Chebyshev distance 2 of ghost g
__device__ __forceinline__ void band_mark_one(const uint32_t *__restrict__ gidx, const uint8_t *__restrict__ cls, const Geo &G,
                              uint8_t *__restrict__ mark, int64_t g) {
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

// Per-level tables: the set-up kernels below process every level of the
// hierarchy in one launch (blocks are assigned to levels by their start
// block), so the many tiny coarse levels do not each pay a serial launch.
struct LevelTab {
    Geo G;
    const double *phi;
    const uint8_t *cls;
    const uint32_t *gidx;
    int64_t ng;
    GhostOut gout;
    uint8_t *mark;
    const uint32_t *bidx;
    int64_t nb;
    int32_t *bref;
    double *bw;
    uint32_t *eg;
    double *ew;
    uint8_t *ecnt;
    uint32_t *eg2;  // second buffer of the expansion passes
    double *ew2;
    uint8_t *ecnt2;
    int64_t blk_g, blk_b;  // first block of this level in the ghost / band launches
};

__device__ __forceinline__ int level_of_block(const LevelTab *tab, int nl, bool band) {
    int l = 0;
    for (int i = 1; i < nl; ++i)
        if ((int64_t)blockIdx.x >= (band ? tab[i].blk_b : tab[i].blk_g)) l = i;
    return l;
}

// ghost geometry and band marks of every level
template <int D>
__global__ void k_ghost_all(const LevelTab *__restrict__ tab, int nl, int bc, int dmode, double dconst, DtauP P) {
    const int l = level_of_block(tab, nl, false);
    const LevelTab &T = tab[l];
    const int64_t g = ((int64_t)blockIdx.x - T.blk_g) * blockDim.x + threadIdx.x;
    if (g >= T.ng) return;
    Geo G = T.G;
    G.d = D;
    ghost_one<D>(bc, T.gidx, T.ng, T.phi, T.cls, G, dmode, dconst, P, T.gout, g);
    band_mark_one(T.gidx, T.cls, G, T.mark, g);
}

__device__ void band_one(const uint32_t *__restrict__ bidx, int64_t nb, const double *__restrict__ phi,
                         const uint8_t *__restrict__ cls, const Geo &G, int32_t *__restrict__ bref,
                         double *__restrict__ bw, int64_t b) {
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

__global__ void k_band_all(const LevelTab *__restrict__ tab, int nl) {
    const int l = level_of_block(tab, nl, true);
    const LevelTab &T = tab[l];
    const int64_t b = ((int64_t)blockIdx.x - T.blk_b) * blockDim.x + threadIdx.x;
    if (b >= T.nb) return;
    band_one(T.bidx, T.nb, T.phi, T.cls, T.G, T.bref, T.bw, b);
}

// The K Jacobi sweeps of the extension, started from zero, are a fixed
// linear map from ghost values to band values.  It is expanded pass by pass,
// as the sweeps run: after pass k the term list of band node b is, over the
// axis sources of b in axis order, the source ghost with its weight w_a, or
// the source band node's list after pass k - 1 scaled by w_a, equal ghosts
// merged (weights summed) in order of first appearance.  At most kExtCap
// terms per band node (ELL layout, term-major); a level with a longer row
// keeps the sweep-by-sweep extension instead.
__global__ void k_ext_pass(const LevelTab *__restrict__ tab, int nl, int d, int first, int last, int to_final,
                           int *__restrict__ overflow) {
    const int l = level_of_block(tab, nl, true);
    const LevelTab &T = tab[l];
    const int64_t b = ((int64_t)blockIdx.x - T.blk_b) * blockDim.x + threadIdx.x;
    if (b >= T.nb) return;
    const int64_t nb = T.nb;
    // the previous pass wrote the other buffer
    const uint8_t *cp = to_final ? T.ecnt2 : T.ecnt;
    const uint32_t *gp = to_final ? T.eg2 : T.eg;
    const double *wp = to_final ? T.ew2 : T.ew;
    uint8_t *co = to_final ? T.ecnt : T.ecnt2;
    uint32_t *go = to_final ? T.eg : T.eg2;
    double *wo = to_final ? T.ew : T.ew2;
    uint32_t g[kExtCap];
    double w[kExtCap];
    int cnt = 0;
    bool over = false;
    auto add = [&](uint32_t gg, double ww) {
        int k = 0;
        while (k < cnt && g[k] != gg) ++k;
        if (k < cnt) w[k] += ww;
        else if (cnt < kExtCap) {
            g[cnt] = gg;
            w[cnt] = ww;
            ++cnt;
        } else {
            over = true;
        }
    };
    for (int ax = 0; ax < d; ++ax) {
        const int32_t ref = T.bref[(int64_t)ax * nb + b];
        if (ref == kNoRef) continue;
        const double wa = T.bw[(int64_t)ax * nb + b];
        if (ref < 0) {
            add((uint32_t)(-(int64_t)ref - 1), wa);
        } else if (!first) {
            const int c = cp[ref];
            for (int k = 0; k < c; ++k) add(gp[(int64_t)k * nb + ref], wa * wp[(int64_t)k * nb + ref]);
        }
    }
    if (over) atomicOr(overflow + l, 1);
    if (last) atomicMax(overflow + nl + l, cnt);  // longest row of the level
    co[b] = (uint8_t)cnt;
    for (int k = 0; k < cnt; ++k) {
        go[(int64_t)k * nb + b] = g[k];
        wo[(int64_t)k * nb + b] = w[k];
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

// derivatives of the Lagrange basis (Neumann rows, Sec. 3.2.2)
__device__ __forceinline__ void lagrange_dw(int q, double xi, double w[3]) {
    w[0] = w[1] = w[2] = 0.0;
    if (q == 2) {
        w[0] = __dsub_rn(xi, 1.5);
        w[1] = __dsub_rn(2.0, __dmul_rn(2.0, xi));
        w[2] = __dsub_rn(xi, 0.5);
    } else if (q == 1) {
        w[0] = -1.0;
        w[1] = 1.0;
    }
}

// Coarsest system: interior rows c u - Lap_h u (eq. Laph), ghost rows the
// boundary operator on the ghost stencil (Dirichlet: tensor Lagrange weights;
// Neumann: sum_a n_a (-s_a / h) L'(xi_a) prod_{b != a} L(xi_b))
__global__ void k_assemble(const uint32_t *__restrict__ act, int64_t nact, const uint8_t *__restrict__ cls,
                           const uint32_t *__restrict__ gidx, const uint16_t *__restrict__ gcode,
                           const double *__restrict__ gxi, const double *__restrict__ gn, int64_t ng, Geo G,
                           int bc, double react, double *__restrict__ A) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nact) return;
    int64_t X = act[r];
    double *row = A + r * nact;
    if (cls[X] == CL_INTERIOR) {
        double ih2 = 1.0 / (G.h * G.h);
        row[r] += 2.0 * G.d * ih2 + react;
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
    double w[3][3] = {{1, 0, 0}, {1, 0, 0}, {1, 0, 0}}, dw[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double nv[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < G.d; ++a) {
        s[a] = ((code >> a) & 1) ? -1 : 1;
        q[a] = (code >> (3 + 2 * a)) & 3;
        lagrange_w(q[a], gxi[(int64_t)a * ng + g], w[a]);
        lagrange_dw(q[a], gxi[(int64_t)a * ng + g], dw[a]);
        nv[a] = gn[(int64_t)a * ng + g];
    }
    for (int o2 = 0; o2 <= q[2]; ++o2)
        for (int o1 = 0; o1 <= q[1]; ++o1)
            for (int o0 = 0; o0 <= q[0]; ++o0) {
                int64_t Y = X - (int64_t)s[0] * o0 * G.st[0] - (int64_t)s[1] * o1 * G.st[1] -
                            (int64_t)s[2] * o2 * G.st[2];
                int64_t c = find_sorted(act, nact, (uint32_t)Y);
                if (c < 0) continue;
                const int o[3] = {o0, o1, o2};
                double v;
                if (bc == BCMG_BC_NEUMANN) {
                    v = 0.0;
                    for (int a = 0; a < G.d; ++a) {
                        double t = __dmul_rn(__dmul_rn(nv[a], __ddiv_rn(-(double)s[a], G.h)), dw[a][o[a]]);
                        for (int b = 0; b < G.d; ++b)
                            if (b != a) t = __dmul_rn(t, w[b][o[b]]);
                        v = __dadd_rn(v, t);
                    }
                } else {
                    v = __dmul_rn(__dmul_rn(w[0][o0], w[1][o1]), w[2][o2]);
                }
                row[c] += v;
            }
}

// Device-to-device copies of several arrays in one launch, in 32-bit words
// (job j: n words from src to dst; blockIdx.y is the job).  Creation copies a
// handful of arrays per level; one launch instead of one driver call each
// keeps concurrent creations from contending for the driver.
struct CopyJob {
    const uint32_t *src;
    uint32_t *dst;
    int64_t n;
};
constexpr int kMaxCopyJobs = 64;
struct CopyBatch {
    int nj;
    CopyJob j[kMaxCopyJobs];
};

__global__ void k_copy_words(CopyBatch B) {
    const CopyJob c = B.j[blockIdx.y];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.n; i += (int64_t)gridDim.x * blockDim.x)
        c.dst[i] = c.src[i];
}

struct Copier {
    Handle &H;
    CopyBatch b{};
    int64_t maxn = 0;
    explicit Copier(Handle &h) : H(h) {}
    // bytes: a multiple of 4; both pointers 4-byte aligned
    void add(const void *src, void *dst, size_t bytes) {
        if (bytes == 0) return;
        if (b.nj == kMaxCopyJobs) flush();
        const int64_t n = (int64_t)(bytes / 4);
        b.j[b.nj++] = CopyJob{(const uint32_t *)src, (uint32_t *)dst, n};
        maxn = std::max(maxn, n);
    }
    void flush() {
        if (b.nj == 0) return;
        const unsigned gx = (unsigned)std::min<int64_t>((maxn + 255) / 256, 1024);
        k_copy_words<<<dim3(gx, (unsigned)b.nj), 256, 0, H.st>>>(b);
        count_launch(H);
        check_cuda(cudaGetLastError(), "array copies");
        b.nj = 0;
        maxn = 0;
    }
};

// the shared-memory limits of the LU kernels are per kernel and device for
// the whole process: set once per device, always to the largest size
void lu_attributes_once();

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

// Small coarsest systems (n <= kLuSmall): LU factorisation with partial
// pivoting (largest |a_ik|, lowest row on ties) of the whole matrix in the
// shared memory of one block, then the columns of the inverse by forward and
// back substitution, one warp per column spread over many SMs (FP64 work on
// one SM is the scarce resource).  PA = LU; row k of the factor holds
// l_k0..l_k,k-1 and u_kk..u_k,n-1; perm[k] is the row swapped into k.
constexpr int kLuSmall = 144;

__global__ void __launch_bounds__(1024) k_lu_small(const double *__restrict__ A, int n, double *__restrict__ LU,
                                                   int *__restrict__ perm, int *__restrict__ singular) {
    extern __shared__ double S[];      // n * n, then the n multipliers of the current column
    double *Lc = S + n * n;
    __shared__ int piv;
    __shared__ double sinv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) S[t] = A[t];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        // 1. pivot (warp 0): largest |a_ik| for i >= k, lowest row on ties,
        //    compared on the bit patterns (integer order is numeric order
        //    for non-negative doubles; no FP64 compares); the reciprocal of
        //    the pivot (one FP64 division per step)
        if (warp == 0) {
            long long best = -1;
            int bidx = n;
            for (int i = k + lane; i < n; i += 32) {
                const long long v = __double_as_longlong(S[i * n + k]) & 0x7fffffffffffffffLL;
                if (v > best) {
                    best = v;
                    bidx = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long v = __shfl_down_sync(0xffffffffu, best, o);
                const int ii = __shfl_down_sync(0xffffffffu, bidx, o);
                if (v > best || (v == best && ii < bidx)) {
                    best = v;
                    bidx = ii;
                }
            }
            if (lane == 0) {
                const bool sing = best <= 0;  // zero column (or nothing left)
                const int pr = sing ? k : bidx;
                piv = pr;
                perm[k] = pr;
                if (sing) *singular = 1;
                sinv = sing ? 0.0 : 1.0 / S[pr * n + k];
            }
        }
        __syncthreads();
        // 2. swap rows k and p; the multipliers l_ik = a_ik / u_kk of the rows
        //    below (row p's old entry is the old a_kk, read by its swapper)
        const int p = piv;
        const double inv = sinv;
        if (p != k)
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const double t = S[k * n + j];
                S[k * n + j] = S[p * n + j];
                S[p * n + j] = t;
                if (j == k) Lc[p] = t * inv;
            }
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x)
            if (i != p) Lc[i] = S[i * n + k] * inv;
        __syncthreads();
        // 3. multipliers into column k and the rank-1 update of the trailing
        //    block, its m x (m + 1) entries dealt out over all threads
        const int m = n - k - 1, w = m + 1;
        for (int t = threadIdx.x; t < m * w; t += blockDim.x) {
            const int i = k + 1 + t / w, jj = t % w;
            if (jj == 0) S[i * n + k] = Lc[i];
            else S[i * n + k + jj] -= Lc[i] * S[k * n + k + jj];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) LU[t] = S[t];
}

// column j of A^-1: solve L U x = P e_j, one warp per column; the block
// first copies the factor into shared memory (every step of the sequential
// substitutions then reads shared memory, not L2) together with the
// reciprocals of U's diagonal (one FP64 division per diagonal entry, not per
// step and lane).  P e_j is a unit vector e_q, so the forward substitution
// starts at row q.
constexpr int kLuColsPerBlock = 4;

__global__ void __launch_bounds__(32 * kLuColsPerBlock) k_lu_inverse(const double *__restrict__ LU, int n,
                                                                     const int *__restrict__ perm,
                                                                     double *__restrict__ Ainv) {
    extern __shared__ double sm[];  // n * n factor, n reciprocals, kLuColsPerBlock * n vectors
    double *F = sm, *rd = sm + n * n;
    // 16-byte copies, several in flight per thread (both buffers are
    // 16-byte aligned: a stream-ordered allocation and dynamic shared memory)
    const int nn = n * n;
    const double2 *src2 = reinterpret_cast<const double2 *>(LU);
    double2 *dst2 = reinterpret_cast<double2 *>(F);
#pragma unroll 4
    for (int t = threadIdx.x; t < nn / 2; t += blockDim.x) dst2[t] = src2[t];
    if ((nn & 1) && threadIdx.x == 0) F[nn - 1] = LU[nn - 1];
    for (int t = threadIdx.x; t < n; t += blockDim.x) rd[t] = 1.0 / LU[t * n + t];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * kLuColsPerBlock + w;
    if (j >= n) return;  // whole warps leave together, after the block barrier
    double *x = sm + n * n + n + w * n;
    // position of e_j after the row swaps of the factorisation
    int q = j;
    for (int k = 0; k < n; ++k) {
        const int p = perm[k];
        if (q == k) q = p;
        else if (q == p) q = k;
    }
    for (int i = lane; i < n; i += 32) x[i] = (i == q) ? 1.0 : 0.0;
    __syncwarp();
    for (int m = q; m < n; ++m) {  // forward: unit lower L (rows above q stay 0)
        const double ym = x[m];
        for (int i = m + 1 + lane; i < n; i += 32) x[i] -= F[i * n + m] * ym;
        __syncwarp();
    }
    for (int m = n - 1; m >= 0; --m) {  // back: upper U
        const double xm = x[m] * rd[m];
        __syncwarp();
        if (lane == 0) x[m] = xm;
        for (int i = lane; i < m; i += 32) x[i] -= F[i * n + m] * xm;
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) Ainv[(int64_t)i * n + j] = x[i];
}

inline int nblocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

double dtau_of(int d, int bc, int mode, double cst, double theta) {
    return dtau_formula(d, bc, mode, cst, theta, dtau_p(d));
}

// the path expansion fits the per-thread buffers: at most d (d^K - 1)/(d - 1)
// the expansion passes work for any number of sweeps (rows longer than
// kExtCap terms fall back per level)
bool ext_ell_ok(int d, int K) { return d >= 1 && K >= 1; }

// ------------------------------------------------------------ batched compaction
// Many flag arrays are compacted with one device->host round trip: block
// counts of every array land in one buffer, the host scans them, offsets go
// back in one copy, then every array is scattered.
namespace {

struct CompactItem {
    const uint8_t *flags;
    int64_t n;
    int nl;                // lists taken from this flag array (1..4)
    uint8_t mask[4];       // list b: the indices with flags & mask[b] != 0
    uint32_t **out[4];     // nullptr: counted only
    bool temp[4];          // list freed when creation ends
    int64_t total[4];
    int64_t nblk = 0, base = 0;
};

CompactItem compact_item(const uint8_t *flags, int64_t n) {
    CompactItem it{};
    it.flags = flags;
    it.n = n;
    return it;
}

void add_list(CompactItem &it, uint8_t mask, uint32_t **out, bool temp) {
    it.mask[it.nl] = mask;
    it.out[it.nl] = out;
    it.temp[it.nl] = temp;
    it.nl++;
}

thread_local int64_t *t_pinned = nullptr;
thread_local size_t t_pinned_n = 0;

// The host scratch of this thread.  Every host write to it follows a stream
// synchronisation, so a copy from it that is still in flight when a set-up
// step returns belongs to the handle being created; before the buffer grows,
// that handle's stream is drained.
int64_t *pinned_scratch(Handle &H, size_t n) {
    if (n > t_pinned_n) {
        check_cuda(cudaStreamSynchronize(H.st), "scratch sync");
        if (t_pinned) cudaFreeHost(t_pinned);
        t_pinned = nullptr;
        t_pinned_n = 0;
        size_t want = std::max<size_t>(n, 1 << 16);
        check_cuda(cudaMallocHost((void **)&t_pinned, want * sizeof(int64_t)), "cudaMallocHost(scratch)");
        t_pinned_n = want;
    }
    return t_pinned;
}

void run_compaction(Handle &H, std::vector<CompactItem> &items) {
    int64_t B = 0;
    for (auto &it : items) {
        it.nblk = std::max<int64_t>((it.n + kCompactTile - 1) / kCompactTile, 1);
        it.base = B;
        B += it.nblk * it.nl;
    }
    if (B == 0) return;
    auto masks_of = [](const CompactItem &it) {
        uint32_t m = 0;
        for (int b = 0; b < it.nl; ++b) m |= (uint32_t)it.mask[b] << (8 * b);
        return m;
    };
    // the arrays in launches of at most kCompactMax
    auto batches = [&](bool with_out, auto &&run) {
        for (size_t i0 = 0; i0 < items.size(); i0 += kCompactMax) {
            CompactBatch cb{};
            int64_t nblk = 0;
            for (size_t i = i0; i < items.size() && i < i0 + kCompactMax; ++i) {
                const CompactItem &it = items[i];
                CompactArr &a = cb.a[cb.narr++];
                a.flags = it.flags;
                a.n = it.n;
                a.blk0 = nblk;
                a.base = it.base;
                a.masks = masks_of(it);
                a.nl = it.nl;
                for (int b = 0; b < it.nl; ++b) a.out[b] = (with_out && it.out[b]) ? *it.out[b] : nullptr;
                nblk += it.nblk;
            }
            run(cb, nblk);
        }
    };
    int64_t *counts = (int64_t *)dalloc(H, sizeof(int64_t) * B, true);
    batches(false, [&](const CompactBatch &cb, int64_t nblk) {
        k_count<<<(unsigned)nblk, kCompactThreads, 0, H.st>>>(cb, counts);
        count_launch(H);
    });
    check_cuda(cudaGetLastError(), "k_count");
    int64_t *hc = pinned_scratch(H, (size_t)B);
    check_cuda(cudaMemcpyAsync(hc, counts, sizeof(int64_t) * B, cudaMemcpyDeviceToHost, H.st), "counts D2H");
    check_cuda(cudaStreamSynchronize(H.st), "compaction sync");
    for (auto &it : items)
        for (int b = 0; b < it.nl; ++b) {
            int64_t tot = 0;
            for (int64_t k = 0; k < it.nblk; ++k) {
                int64_t &slot = hc[it.base + k * it.nl + b];
                const int64_t c = slot;
                slot = tot;
                tot += c;
            }
            it.total[b] = tot;
        }
    check_cuda(cudaMemcpyAsync(counts, hc, sizeof(int64_t) * B, cudaMemcpyHostToDevice, H.st), "offsets H2D");
    for (auto &it : items)
        for (int b = 0; b < it.nl; ++b)
            if (it.out[b])
                *it.out[b] = (uint32_t *)dalloc(H, sizeof(uint32_t) * (size_t)std::max<int64_t>(it.total[b], 1),
                                                it.temp[b], false);
    batches(true, [&](const CompactBatch &cb, int64_t nblk) {
        k_scatter<<<(unsigned)nblk, kCompactThreads, 0, H.st>>>(cb, counts);
        count_launch(H);
    });
    check_cuda(cudaGetLastError(), "k_scatter");
}

// hyperplane (p = i + j + k) of each interior node: counts, then positions
__global__ void k_hp_count(const uint32_t *__restrict__ ilist, int64_t nint, Geo G, int *__restrict__ counts) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nint) return;
    int ix[3];
    decode(G, ilist[t], ix);
    atomicAdd(counts + ix[0] + ix[1] + ix[2], 1);
}

// within a hyperplane the order does not matter: its nodes are not
// neighbours of one another
__global__ void k_hp_scatter(const uint32_t *__restrict__ ilist, int64_t nint, Geo G, int *__restrict__ cursor,
                             uint32_t *__restrict__ hlist) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nint) return;
    const uint32_t X = ilist[t];
    int ix[3];
    decode(G, X, ix);
    hlist[atomicAdd(cursor + ix[0] + ix[1] + ix[2], 1)] = X;
}

struct LevelScratch {
    uint8_t *flags = nullptr, *fband = nullptr;
    uint32_t *red = nullptr, *black = nullptr;
    uint32_t *act = nullptr;  // active list of a coarse level (pass 1)
    int64_t nact = 0;
    unsigned long long *cnt = nullptr;  // clamp / fall-back counters
    int64_t *ecnt = nullptr;
};

}  // namespace

// Build every level of the hierarchy (Sec. 2.1 re-discretisation, Sec. 3.3
// geometry).  Four host synchronisations in total.
void setup_hierarchy(Handle &H, const double *phi0) {
    const int T = 256;
    // candidate levels: N_l = N / 2^l while N_l is even and N_l / 2 >= min_coarse
    {
        int64_t Nl = H.N;
        for (int l = 0; l < H.o.max_levels; ++l) {
            Level L;
            L.d = H.d;
            L.N = (int)Nl;
            L.n = (int)Nl + 1;
            // h_l = h_0 2^l (exact: a power-of-two scaling)
            L.h = std::ldexp(H.h0, l);
            L.lo = H.lo;
            L.react = H.o.reaction;
            L.nn = 1;
            for (int a = 0; a < H.d; ++a) {
                L.st[a] = L.nn;
                L.nn *= L.n;
            }
            L.lay.s = L.lay.m = 1;
            L.lay.ho = (uint32_t)split_ho(L.nn);
            H.L.push_back(L);
            if (Nl % 2 != 0 || Nl / 2 < H.o.min_coarse) break;
            Nl /= 2;
        }
    }
    const int nc = (int)H.L.size();
    std::vector<LevelScratch> S(nc);
    // phase A: phi by injection, classes and class flags (one launch per
    // kClassMax levels)
    {
        ClassBatch cb{};
        int64_t nblk = 0;
        auto flush = [&]() {
            if (cb.nl == 0) return;
            if (H.d == 3) k_classify<3><<<(unsigned)nblk, dim3(32, 4), 0, H.st>>>(cb);
            else k_classify<2><<<(unsigned)nblk, dim3(32, 4), 0, H.st>>>(cb);
            count_launch(H);
            check_cuda(cudaGetLastError(), "classification");
            cb.nl = 0;
            nblk = 0;
        };
        const Geo G0 = geo_of(H.L[0]);
        for (int l = 0; l < nc; ++l) {
            Level &L = H.L[l];
            LevelScratch &s = S[l];
            Geo G = geo_of(L);
            double *phic = l == 0 ? nullptr : (double *)dalloc(H, sizeof(double) * L.nn, true, false);
            L.phi = l == 0 ? phi0 : phic;
            L.cls = (uint8_t *)dalloc(H, L.nn, false, false);  // k_classify writes every entry
            s.flags = (uint8_t *)dalloc(H, (size_t)L.nn, true, false);
            if (cb.nl == kClassMax) flush();
            cb.phi0 = phi0;
            for (int a = 0; a < 3; ++a) cb.st0[a] = G0.st[a];
            ClassLevel &c = cb.lv[cb.nl++];
            c.G = G;
            c.s = 1 << l;
            c.phic = phic;
            c.cls = L.cls;
            c.flags = s.flags;
            c.blk0 = nblk;
            c.bx = nblocks(L.n, 32);
            c.by = nblocks(L.n, 4);
            nblk += (int64_t)c.bx * c.by * (H.d == 3 ? nblocks(L.n, kClassPlanes) : 1);
        }
        flush();
    }
    // pass 1: counts of every list on every candidate level (one sync)
    {
        std::vector<CompactItem> items;
        for (int l = 0; l < nc; ++l) {
            Level &L = H.L[l];
            LevelScratch &s = S[l];
            CompactItem it = compact_item(s.flags, L.nn);
            add_list(it, kFlRed, &s.red, true);
            add_list(it, kFlBlack, &s.black, true);
            add_list(it, kFlBox, l == 0 ? &L.boxidx : nullptr, false);
            add_list(it, kFlGhost, &L.gidx, false);
            items.push_back(it);
        }
        // the active list of every coarse level (small), so that the
        // coarsest system can be set up as soon as its ghosts are
        for (int l = 1; l < nc; ++l) {
            CompactItem it = compact_item(S[l].flags, H.L[l].nn);
            add_list(it, kFlAct, &S[l].act, true);
            items.push_back(it);
        }
        for (int l = 0; l < nc; ++l) {
            CompactItem it = compact_item(S[l].flags, H.L[l].nn);
            add_list(it, kFlBNear, &H.L[l].bnear, false);
            items.push_back(it);
        }
        run_compaction(H, items);
        for (int l = 0; l < nc; ++l) {
            Level &L = H.L[l];
            L.nred = items[l].total[0];
            L.nbn = items[2 * nc - 1 + l].total[0];
            L.nint = L.nred + items[l].total[1];
            L.nbox = items[l].total[2];
            L.ng = items[l].total[3];
            if (l > 0) S[l].nact = items[nc + l - 1].total[0];
        }
    }
    if (H.L[0].nint == 0) throw Error{BCMG_EGEOM, "no interior node on the finest grid"};
    int keep = nc;
    for (int l = 1; l < nc; ++l)
        if (H.L[l].nint == 0) {
            keep = l;
            break;
        }
    H.L.resize(keep);
    S.resize(keep);
    // coarsest: dense system and its inverse, on the side stream (one SM's
    // work for small systems) while the main stream goes on with the set-up;
    // needs the coarsest active list and ghost geometry; joined before
    // creation's closing synchronisation
    auto coarsest_on_side = [&]() {
        Level &L = H.L[keep - 1];
        Geo G = geo_of(L);
        int64_t n = L.nact;
        double *A = (double *)dalloc(H, sizeof(double) * std::max<int64_t>(n * n, 1), true);
        L.Ainv = (double *)dalloc(H, sizeof(double) * std::max<int64_t>(n * n, 1));
        L.crhs = (double *)dalloc(H, sizeof(double) * std::max<int64_t>(n, 1));
        double *col = (double *)dalloc(H, sizeof(double) * std::max<int64_t>(n, 1), true);
        int *sing = (int *)dalloc(H, sizeof(int), true);
        double *LU = nullptr;
        int *perm = nullptr;
        if (n <= kLuSmall) {
            LU = (double *)dalloc(H, sizeof(double) * std::max<int64_t>(n * n, 1), true);
            perm = (int *)dalloc(H, sizeof(int) * std::max<int64_t>(n, 1), true);
        }
        // every buffer above (and the level data it reads) is in place on the
        // main stream before the side stream starts
        check_cuda(cudaEventRecord(H.ev_fork, H.st), "fork record");
        check_cuda(cudaStreamWaitEvent(H.st2, H.ev_fork, 0), "fork wait");
        k_assemble<<<nblocks(n, 128), 128, 0, H.st2>>>(L.act, n, L.cls, L.gidx, L.gcode, L.gxi, L.gn, L.ng, G, H.o.bc,
                                                      H.o.reaction, A);
        count_launch(H);
        if (n <= kLuSmall) {
            // shared-memory limits are per kernel for the whole process: always
            // the largest size (n = kLuSmall), never one handle's n
            const size_t smem = sizeof(double) * (size_t)(n * n + n);
            lu_attributes_once();
            k_lu_small<<<1, 1024, smem, H.st2>>>(A, (int)n, LU, perm, sing);
            count_launch(H);
            const size_t smem2 = sizeof(double) * (size_t)(n * n + n + kLuColsPerBlock * n);
            k_lu_inverse<<<nblocks(n, kLuColsPerBlock), 32 * kLuColsPerBlock, smem2, H.st2>>>(LU, (int)n, perm, L.Ainv);
            count_launch(H);
        } else {
            k_identity<<<nblocks(n * n, T), T, 0, H.st2>>>(L.Ainv, n);
            count_launch(H);
            for (int64_t k = 0; k < n; ++k) {
                k_gj_pivot<<<1, 1024, 0, H.st2>>>(A, L.Ainv, n, k, col, sing);
                k_gj_elim<<<nblocks(n * n, T), T, 0, H.st2>>>(A, L.Ainv, n, k, col);
                count_launch(H);
                count_launch(H);
            }
        }
        check_cuda(cudaGetLastError(), "gauss-jordan");
        // into the handle's own pinned block, read after creation's closing
        // synchronisation
        check_cuda(cudaMemcpyAsync(H.sing_host, sing, sizeof(int), cudaMemcpyDeviceToHost, H.st2), "singular flag");
        check_cuda(cudaEventRecord(H.ev_join, H.st2), "join record");
    };
    // phase B: interior lists and ghost arrays per level, then the ghost geometry
    // and band marks of every level in one launch
    std::vector<LevelTab> tab(keep);
    int64_t gblocks = 0;
    Copier lists(H);
    // the band marks of every level: slices of one zero-filled block
    size_t fb_bytes = 0;
    for (int l = 0; l < keep; ++l) fb_bytes += ((size_t)H.L[l].nn + 255) & ~(size_t)255;
    uint8_t *fb_next = (uint8_t *)dalloc(H, fb_bytes, true);
    // the ghost counters of every level (two each) and the extension's
    // overflow flags and longest rows (two ints per level), contiguous, so
    // that pass 3 reads them back with one copy
    char *ctr = (char *)dalloc(H, (sizeof(unsigned long long) * 2 + sizeof(int) * 2) * (size_t)keep, true);
    for (int l = 0; l < keep; ++l) {
        Level &L = H.L[l];
        LevelScratch &s = S[l];
        Geo G = geo_of(L);
        // arrays every entry of which a set-up kernel or copy writes take
        // no zero-fill
        L.ilist = (uint32_t *)dalloc(H, sizeof(uint32_t) * (size_t)std::max<int64_t>(L.nint, 1), false, false);
        lists.add(s.red, L.ilist, sizeof(uint32_t) * (size_t)L.nred);
        lists.add(s.black, L.ilist + L.nred, sizeof(uint32_t) * (size_t)(L.nint - L.nred));
        int64_t ng1 = std::max<int64_t>(L.ng, 1);
        L.gcode = (uint16_t *)dalloc(H, sizeof(uint16_t) * ng1, false, false);
        L.gxi = (double *)dalloc(H, sizeof(double) * 3 * ng1);
        L.gn = (double *)dalloc(H, sizeof(double) * 3 * ng1);
        L.gdt = (double *)dalloc(H, sizeof(double) * ng1, false, false);
        L.geta = (double *)dalloc(H, sizeof(double) * ng1, false, false);
        L.gQ = (double *)dalloc(H, sizeof(double) * 3 * ng1);
        L.gtmp = (double *)dalloc(H, sizeof(double) * ng1, false, false);
        s.cnt = (unsigned long long *)ctr + 2 * l;
        s.fband = fb_next;  // zero-filled
        fb_next += ((size_t)L.nn + 255) & ~(size_t)255;
        LevelTab &t = tab[l];
        t = LevelTab{};
        t.G = G;
        t.phi = L.phi;
        t.cls = L.cls;
        t.gidx = L.gidx;
        t.ng = L.ng;
        t.gout = GhostOut{L.gcode, L.gxi, L.gdt, L.geta, L.gn, L.gQ, s.cnt, s.cnt + 1};
        t.mark = s.fband;
        t.blk_g = gblocks;
        gblocks += nblocks(L.ng, 128);
    }
    lists.flush();
    // which black entries are listed apart (one bit each, from the flags)
    {
        if (keep > kNearMax) throw Error{BCMG_EINVAL, "too many levels"};
        NearBatch nbt{};
        int64_t blk = 0;
        for (int l = 0; l < keep; ++l) {
            Level &L = H.L[l];
            const int64_t nb = L.nint - L.nred;
            L.bmask =
                (uint32_t *)dalloc(H, sizeof(uint32_t) * (size_t)std::max<int64_t>((nb + 31) / 32, 1), false, false);
            nbt.lv[nbt.nl++] = NearLevel{L.ilist + L.nred, S[l].flags, L.bmask, nb, blk};
            blk += nblocks(nb, 256);
        }
        if (blk > 0) {
            k_near_bits<<<(unsigned)blk, 256, 0, H.st>>>(nbt);
            count_launch(H);
        }
        check_cuda(cudaGetLastError(), "k_near_bits");
    }
    LevelTab *tab_d = (LevelTab *)dalloc(H, sizeof(LevelTab) * keep, true);
    check_cuda(cudaMemcpyAsync(tab_d, tab.data(), sizeof(LevelTab) * keep, cudaMemcpyHostToDevice, H.st), "tab");
    if (gblocks > 0) {
        if (H.d == 3)
            k_ghost_all<3><<<(unsigned)gblocks, 128, 0, H.st>>>(tab_d, keep, H.o.bc, H.o.dtau_mode, H.o.dtau_const,
                                                                 dtau_p(H.d));
        else
            k_ghost_all<2><<<(unsigned)gblocks, 128, 0, H.st>>>(tab_d, keep, H.o.bc, H.o.dtau_mode, H.o.dtau_const,
                                                                 dtau_p(H.d));
        count_launch(H);
    }
    check_cuda(cudaGetLastError(), "ghost set-up");
    Level &Lc = H.L[keep - 1];
    if (keep > 1) {
        // a coarse level is the coarsest: its active list is there
        Lc.nact = S[keep - 1].nact;
        if (Lc.nact > kMaxCoarse) throw Error{BCMG_EGEOM, "coarsest system has more than 4096 unknowns"};
        Lc.act = (uint32_t *)dalloc(H, sizeof(uint32_t) * (size_t)std::max<int64_t>(Lc.nact, 1), false, false);
        if (Lc.nact > 0)
            check_cuda(cudaMemcpyAsync(Lc.act, S[keep - 1].act, sizeof(uint32_t) * Lc.nact, cudaMemcpyDeviceToDevice,
                                       H.st),
                       "active list");
        coarsest_on_side();
    }
    // pass 2: band lists on every level (and the active list of a finest
    // level that is also the coarsest) (one sync)
    {
        std::vector<CompactItem> items;
        for (int l = 0; l < keep; ++l) {
            CompactItem it = compact_item(S[l].fband, H.L[l].nn);
            add_list(it, 0xff, &H.L[l].bidx, false);
            items.push_back(it);
        }
        if (keep == 1) {
            CompactItem ia = compact_item(S[0].flags, Lc.nn);
            add_list(ia, kFlAct, &Lc.act, false);
            items.push_back(ia);
        }
        run_compaction(H, items);
        for (int l = 0; l < keep; ++l) H.L[l].nb = items[l].total[0];
        if (keep == 1) Lc.nact = items[keep].total[0];
    }
    if (keep == 1) {
        if (Lc.nact > kMaxCoarse) throw Error{BCMG_EGEOM, "coarsest system has more than 4096 unknowns"};
        coarsest_on_side();
    }
    // phase C: band sources and the ELL expansion of the extension, every
    // level in one launch each
    const bool ell = ext_ell_ok(H.d, H.o.ext_sweeps);
    int64_t bblocks = 0;
    int *ovf = (int *)(ctr + sizeof(unsigned long long) * 2 * keep);  // overflow flags, longest rows
    for (int l = 0; l < keep; ++l) {
        Level &L = H.L[l];
        int64_t nb1 = std::max<int64_t>(L.nb, 1);
        L.bref = (int32_t *)dalloc(H, sizeof(int32_t) * 3 * nb1, false, false);
        L.bw = (double *)dalloc(H, sizeof(double) * 3 * nb1, false, false);
        L.bbuf = (double *)dalloc(H, sizeof(double) * 2 * nb1, false, false);
        if (ell && L.nb > 0) {
            L.ecnt = (uint8_t *)dalloc(H, (size_t)nb1, false, false);
            // expansion scratch with kExtCap slots; the resident copy keeps
            // only the slots the level's longest row needs (see pass 3)
            L.eg = (uint32_t *)dalloc(H, sizeof(uint32_t) * kExtCap * nb1, true, false);
            L.ew = (double *)dalloc(H, sizeof(double) * kExtCap * nb1, true, false);
        }
        LevelTab &t = tab[l];
        t.bidx = L.bidx;
        t.nb = L.nb;
        t.bref = L.bref;
        t.bw = L.bw;
        t.eg = L.eg;
        t.ew = L.ew;
        t.ecnt = L.ecnt;
        if (ell && L.nb > 0) {
            t.ecnt2 = (uint8_t *)dalloc(H, (size_t)nb1, true, false);
            t.eg2 = (uint32_t *)dalloc(H, sizeof(uint32_t) * kExtCap * nb1, true, false);
            t.ew2 = (double *)dalloc(H, sizeof(double) * kExtCap * nb1, true, false);
        }
        t.blk_b = bblocks;
        bblocks += nblocks(L.nb, 128);
    }
    check_cuda(cudaMemcpyAsync(tab_d, tab.data(), sizeof(LevelTab) * keep, cudaMemcpyHostToDevice, H.st), "tab");
    if (bblocks > 0) {
        k_band_all<<<(unsigned)bblocks, 128, 0, H.st>>>(tab_d, keep);
        count_launch(H);
        if (ell) {
            // pass k writes the final buffer when K - k is even, so the last
            // pass (k = K) lands in it
            const int K = H.o.ext_sweeps;
            for (int k = 1; k <= K; ++k) {
                k_ext_pass<<<(unsigned)bblocks, 128, 0, H.st>>>(tab_d, keep, H.d, k == 1, k == K, (K - k) % 2 == 0,
                                                                 ovf);
                count_launch(H);
            }
        }
    }
    check_cuda(cudaGetLastError(), "band set-up");
    // pass 3: clamp / fall-back counters and ELL overflows (one sync)
    {
        int64_t *hc = pinned_scratch(H, 3 * (size_t)keep + 2);
        check_cuda(cudaMemcpyAsync(hc, ctr, (sizeof(int64_t) * 2 + sizeof(int) * 2) * (size_t)keep,
                                   cudaMemcpyDeviceToHost, H.st),
                   "ghost counters, overflow");
        int *hov = (int *)(hc + 2 * keep);
        check_cuda(cudaStreamSynchronize(H.st), "set-up sync 3");
        Copier ell(H);
        // term-major ELL: the first ell_max slabs are the whole map; keep a
        // multiple of 8 slots (the tail reads 8-term rounds), the extra slots
        // zero -- the kept maps of every level are slices of one zero-filled
        // block
        auto slots_of = [&](const Level &L) { return std::min(kExtCap, ((std::max(L.ell_max, 1) + 7) / 8) * 8); };
        auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
        size_t ebytes = 0;
        for (int l = 0; l < keep; ++l) {
            Level &L = H.L[l];
            L.nclamp = hc[2 * l];
            L.nfall = hc[2 * l + 1];
            if (hov[l]) L.ecnt = nullptr;  // a row longer than kExtCap: sweep by sweep
            L.ell_max = hov[keep + l];
            if (L.ecnt) {
                const size_t nb1 = (size_t)std::max<int64_t>(L.nb, 1);
                ebytes += al(sizeof(uint32_t) * slots_of(L) * nb1) + al(sizeof(double) * slots_of(L) * nb1);
            }
        }
        char *enext = ebytes > 0 ? (char *)dalloc(H, ebytes) : nullptr;
        for (int l = 0; l < keep; ++l) {
            Level &L = H.L[l];
            if (L.ecnt) {
                const int64_t nb1 = std::max<int64_t>(L.nb, 1);
                const int slots = slots_of(L);
                uint32_t *eg = (uint32_t *)enext;
                enext += al(sizeof(uint32_t) * slots * nb1);
                double *ew = (double *)enext;
                enext += al(sizeof(double) * slots * nb1);
                ell.add(L.eg, eg, sizeof(uint32_t) * (size_t)L.ell_max * nb1);
                ell.add(L.ew, ew, sizeof(double) * (size_t)L.ell_max * nb1);
                L.eg = eg;
                L.ew = ew;
            }
        }
        ell.flush();
    }
    // GS-LEX: interior nodes grouped by hyperplane on every level (one sync)
    if (H.o.ordering == BCMG_ORDER_LEX) {
        std::vector<int *> cnt(keep);
        std::vector<int64_t> base(keep + 1, 0);
        for (int l = 0; l < keep; ++l) base[l + 1] = base[l] + (int64_t)H.d * H.L[l].N + 1;
        int *counts = (int *)dalloc(H, sizeof(int) * base[keep], true);
        for (int l = 0; l < keep; ++l) {
            Level &L = H.L[l];
            if (L.nint > 0) {
                k_hp_count<<<nblocks(L.nint, T), T, 0, H.st>>>(L.ilist, L.nint, geo_of(L), counts + base[l]);
                count_launch(H);
            }
        }
        int64_t *hc = pinned_scratch(H, (size_t)base[keep]);
        int *hci = (int *)hc;
        check_cuda(cudaMemcpyAsync(hci, counts, sizeof(int) * base[keep], cudaMemcpyDeviceToHost, H.st), "hp counts");
        check_cuda(cudaStreamSynchronize(H.st), "hp sync");
        std::vector<int> cursor((size_t)base[keep]);
        for (int l = 0; l < keep; ++l) {
            Level &L = H.L[l];
            const int64_t np = base[l + 1] - base[l];
            L.hoff.assign((size_t)np + 1, 0);
            for (int64_t q = 0; q < np; ++q) {
                cursor[base[l] + q] = (int)L.hoff[q];
                L.hoff[q + 1] = L.hoff[q] + hci[base[l] + q];
            }
        }
        check_cuda(cudaMemcpyAsync(counts, cursor.data(), sizeof(int) * base[keep], cudaMemcpyHostToDevice, H.st),
                   "hp cursor");
        for (int l = 0; l < keep; ++l) {
            Level &L = H.L[l];
            L.hlist = (uint32_t *)dalloc(H, sizeof(uint32_t) * (size_t)std::max<int64_t>(L.nint, 1));
            if (L.nint > 0) {
                k_hp_scatter<<<nblocks(L.nint, T), T, 0, H.st>>>(L.ilist, L.nint, geo_of(L), counts + base[l],
                                                                 L.hlist);
                count_launch(H);
            }
        }
        check_cuda(cudaGetLastError(), "hyperplanes");
        // the pageable cursor copy must be done before the vector goes
        check_cuda(cudaStreamSynchronize(H.st), "hp sync 2");
    }
    // level arrays: value arrays in the parity-split layout (split_len
    // entries).  Those that must start at zero -- u of the coarse levels, F
    // of the finest (it keeps zeros until the caller sets its data; coarse
    // levels get every row they read from the restriction), r, and their
    // FP32 copies -- are slices of one zero-filled block (one allocation and
    // one fill for the whole hierarchy); the others are written before they
    // are read.
    const bool mixed = H.o.precision == BCMG_PREC_MIXED;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t zbytes = 0;
    for (int l = 0; l < keep; ++l) {
        const size_t sl = (size_t)split_len(H.L[l].nn);
        zbytes += 2 * al(sizeof(double) * sl);                  // u (coarse) or F (finest), and r
        if (mixed) zbytes += 2 * al(sizeof(float) * sl);        // u32, r32
    }
    char *z = (char *)dalloc(H, zbytes);
    auto take = [&](size_t b) {
        char *p = z;
        z += al(b);
        return p;
    };
    for (int l = 0; l < keep; ++l) {
        Level &L = H.L[l];
        const int64_t sl = split_len(L.nn);
        if (l > 0) {
            L.u = (double *)take(sizeof(double) * sl);
            L.F = (double *)dalloc(H, sizeof(double) * sl, false, false);
        } else {
            L.F = (double *)take(sizeof(double) * sl);
        }
        L.Fs = (double *)dalloc(H, sizeof(double) * sl, false, false);
        L.r = (double *)take(sizeof(double) * sl);
        if (mixed) {
            L.u32 = (float *)take(sizeof(float) * sl);
            L.F32 = (float *)dalloc(H, sizeof(float) * sl, false, false);
            L.Fs32 = (float *)dalloc(H, sizeof(float) * sl, false, false);
            L.r32 = (float *)take(sizeof(float) * sl);
            L.gtmp32 = (float *)dalloc(H, sizeof(float) * std::max<int64_t>(L.ng, 1));
            L.bbuf32 = (float *)dalloc(H, sizeof(float) * 2 * std::max<int64_t>(L.nb, 1));
        }
    }
}

}  // namespace bcmg

namespace bcmg {
namespace {
std::mutex g_lu_attr_mu;
std::set<int> g_lu_attr_devs;

void lu_attributes_once() {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_lu_attr_mu);
    if (g_lu_attr_devs.count(dev)) return;
    check_cuda(cudaFuncSetAttribute(k_lu_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(double) * (kLuSmall * kLuSmall + kLuSmall))),
               "LU shared memory");
    check_cuda(cudaFuncSetAttribute(k_lu_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(double) * (kLuSmall * kLuSmall + (2 + kLuColsPerBlock) * kLuSmall))),
               "LU inverse shared memory");
    g_lu_attr_devs.insert(dev);
}
}  // namespace
}  // namespace bcmg
