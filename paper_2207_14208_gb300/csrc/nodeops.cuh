// Per-node steps of the BCMG cycle (arXiv 2207.14208) shared by the
// single-hierarchy kernels (cycle.cu) and the batched ones (batch.cu): the
// grid-constant block G2, the programmatic-launch helpers, and the device
// functions that update, relax, restrict, prolong or extend one node.  Both
// translation units run exactly this arithmetic, so a node computed in a
// batch is the same as one computed alone.
#pragma once

#include "bcmg_internal.cuh"

namespace bcmg {
namespace {

struct G2 {
    int d, N, n;
    int64_t sy, sz;
    Lay lay;  // layout of the level's value arrays
    double h2, ih2;
    double diag, inv_diag;  // 2d + c h^2 of c u - Lap_h u = f, and its inverse
};

G2 g2_of(const Level &L) {
    G2 g;
    g.d = L.d;
    g.N = L.N;
    g.n = L.n;
    g.sy = L.st[1];
    g.sz = L.st[2];
    g.lay = L.lay;
    g.h2 = L.h * L.h;
    g.ih2 = 1.0 / g.h2;
    g.diag = 2.0 * L.d + L.react * g.h2;  // exactly 2d without reaction
    g.inv_diag = 1.0 / g.diag;
    return g;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
constexpr int kT = 256;           // largest block of the grid kernels
constexpr int kMultiMin = 2048;   // sweeps with more entries per SM than this
                                  // take several entries per thread (FP32)
constexpr int kTailThreads = 512; // threads per CTA of the cluster tail

// block size for n independent work items: the largest of 256, 128, 64 that
// still gives every SM about four blocks (FP64 work is spread, not queued)
int bs_for(const Handle &H, int64_t n) {
    int bs = kT;
    while (bs > 64 && (int64_t)nblk(n, bs) < 4 * (int64_t)H.nsm) bs >>= 1;
    return bs;
}

// Programmatic dependent launch: every cycle kernel is launched with
// programmatic stream serialisation, so its CTAs may be scheduled while its
// predecessor drains; each kernel waits (griddepcontrol.wait: per the PTX ISA
// it returns once the prerequisite grid has completed and its memory
// operations are performed and made visible to the waiting grid) and then
// allows its own successor to be scheduled (griddepcontrol.launch_dependents).
// Before the wait a kernel reads the level tables that are fixed once the
// hierarchy exists (node lists, ghost codes, weights and steps, class bytes,
// family masks, extension maps; creation ends with a stream
// synchronisation), and three kernels also do part of their work: the ghost
// rows of a residual, the coarse interior rows of a restriction and the
// prolongation of rows with no band corner.  That work reads only values
// written by grids two or more launches back and writes only what its
// predecessor neither reads nor writes.  Why those values are visible: a
// kernel's CTAs are launched only after every CTA of its predecessor has
// executed launch_dependents, which each does right after its own wait, so
// the grid two back has completed and its writes were performed and made
// visible to the predecessor's threads on every SM -- device scope, whose
// point of coherence is L2 -- before this kernel starts.  The early work reads
// those values with ld.global.cg, which caches in L2 and not in L1, so no SM
// can serve it a line cached before they were written.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename K, typename... A>
void launch(Handle &H, const char *name, K kern, unsigned grid, unsigned block, A... args) {
    if (grid == 0) return;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = H.st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    check_cuda(cudaLaunchKernelEx(&cfg, kern, args...), name);
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

__device__ __forceinline__ void coords(uint32_t X, uint32_t n, int D, int ic[3]) {
    const uint32_t q = X / n;
    ic[0] = (int)(X - q * n);
    if (D == 3) {
        const uint32_t q2 = q / n;
        ic[1] = (int)(q - q2 * n);
        ic[2] = (int)q2;
    } else {
        ic[1] = (int)q;
        ic[2] = 0;
    }
}

// Loads of values a cycle writes.  CG = false: ordinary loads (after the
// dependency wait).  CG = true: ld.global.cg, cached in L2 only, for the work
// a few kernels do before their wait on data that grids two or more
// launches back wrote (see pdl_begin): L2 is the device-wide point of
// coherence, so those loads cannot hit a stale line of an SM's L1.
template <bool CG, typename T>
__device__ __forceinline__ T ldv(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// B u~ at a ghost: the (tri/bi)quadratic interpolant on ST_G at Q (eq. BCh),
// with the tensor-product Lagrange weights tabulated per ghost (gw, term
// (o2 * 3 + o1) * 3 + o0, term-major).  Branch-free: every term's loads are
// predicated on the term lying within the stencil's degrees, so all of them
// are in flight together; one partial sum per stencil row.
template <int D>
__device__ __forceinline__ bool ghost_term(uint16_t code, int k) {
    const int qx = (code >> 3) & 3, qy = (code >> 5) & 3, qz = (D == 3) ? ((code >> 7) & 3) : 0;
    return k % 3 <= qx && (k / 3) % 3 <= qy && k / 9 <= qz;
}

// the ghost's tabulated weights (zero outside the stencil's degrees)
template <int D, typename T>
__device__ __forceinline__ void ghost_weights(uint16_t code, const T *gw, int64_t ng, int64_t g,
                                              T w[(D == 3) ? 27 : 9]) {
#pragma unroll
    for (int k = 0; k < ((D == 3) ? 27 : 9); ++k) w[k] = ghost_term<D>(code, k) ? gw[(int64_t)k * ng + g] : T(0);
}

template <int D, typename T, bool CG = false>
__device__ __forceinline__ T ghost_Bw(int64_t X, uint16_t code, const T *w, const T *u, const G2 &G) {
    const int64_t ox = (code & 1) ? 1 : -1;
    const int64_t oy = (code & 2) ? G.sy : -G.sy;
    const int64_t oz = (D == 3) ? ((code & 4) ? G.sz : -G.sz) : 0;
    constexpr int NT = (D == 3) ? 27 : 9;
    T v[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        const int o0 = k % 3, o1 = (k / 3) % 3, o2 = k / 9;
        v[k] = ghost_term<D>(code, k) ? ldv<CG>(u + pos(X + o2 * oz + o1 * oy + o0 * ox, G.lay)) : T(0);
    }
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int k = 0; k < NT; ++k) acc[(k / 3) % 3] = fma(w[k], v[k], acc[(k / 3) % 3]);
    return (acc[0] + acc[1]) + acc[2];
}

// One stencil row of B u~ (the terms with outermost offset `row`: o2 in 3D,
// o1 in 2D), for lanes that share a ghost; B u~ is the sum of the rows
template <int D, typename T>
__device__ __forceinline__ T ghost_row(int64_t X, uint16_t code, const T *gw, int64_t ng, int64_t g, const T *u,
                                       const G2 &G, int row) {
    const int64_t ox = (code & 1) ? 1 : -1;
    const int64_t oy = (code & 2) ? G.sy : -G.sy;
    const int64_t oz = (D == 3) ? ((code & 4) ? G.sz : -G.sz) : 0;
    constexpr int NR = (D == 3) ? 9 : 3;
    const int64_t base = X + (D == 3 ? row * oz : row * oy);
    T w[NR], v[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int k = row * NR + j;
        const int o0 = j % 3, o1 = (D == 3) ? j / 3 : 0;
        const bool p = ghost_term<D>(code, k);
        w[j] = p ? gw[(int64_t)k * ng + g] : T(0);
        v[j] = p ? u[pos(base + o1 * oy + o0 * ox, G.lay)] : T(0);
    }
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < NR; ++j) acc = fma(w[j], v[j], acc);
    return acc;
}

// B u~ of the ghost shared by the four lanes of a group (lane sub < 3 takes
// row sub, lane 3 none); every lane of the warp must call it; all four get
// the sum
template <int D, typename T>
__device__ __forceinline__ T ghost_B4(bool on, int sub, int64_t X, uint16_t code, const T *gw, int64_t ng,
                                      int64_t g, const T *u, const G2 &G) {
    T part = (on && sub < 3) ? ghost_row<D, T>(X, code, gw, ng, g, u, G, sub) : T(0);
    part += __shfl_xor_sync(0xffffffffu, part, 1);
    part += __shfl_xor_sync(0xffffffffu, part, 2);
    return part;
}

template <int D, typename T>
__device__ __forceinline__ T nbr_sum(const T *u, int64_t X, const G2 &G) {
    T s = (u[pos(X - 1, G.lay)] + u[pos(X + 1, G.lay)]) + (u[pos(X - G.sy, G.lay)] + u[pos(X + G.sy, G.lay)]);
    if (D == 3) s += u[pos(X - G.sz, G.lay)] + u[pos(X + G.sz, G.lay)];
    return s;
}

// ------------------------------------------------------------ per-node steps
// red-black Gauss-Seidel update of interior node X (eq. GSLEX_2D in
// red-black order) of c u - Lap_h u = f: u_X = (sum of 2d neighbours +
// h^2 F_X) / (2d + c h^2)
template <int D, typename T>
__device__ __forceinline__ void smooth_at(int64_t X, T *u, const T *F, const G2 &G) {
    const T s = nbr_sum<D, T>(u, X, G);
    const int64_t x = pos(X, G.lay);
    u[x] = fma((T)G.h2, F[x], s) * (T)G.inv_diag;
}

// the same update from Fs = h^2 F / (2d + c h^2), kept beside F on the
// cycle's interior rows: s / diag + Fs, one FP64 instruction fewer
template <int D, typename T>
__device__ __forceinline__ void smooth_at_s(int64_t X, T *u, const T *Fs, const G2 &G) {
    const T s = nbr_sum<D, T>(u, X, G);
    const int64_t x = pos(X, G.lay);
    u[x] = fma(s, (T)G.inv_diag, Fs[x]);
}

// The same update when every node of the list has the parity par of its
// index and n is odd (the red and black lists of every smoothed level): with
// m = X >> 1 the node sits at m in its own half and its 2d neighbours, all
// of the other parity, at fixed offsets from m in the other half, so the
// sweep reads one contiguous run of the other colour per axis direction and
// writes its own colour densely.  Same terms, same order as nbr_sum.
template <int D, typename T>
__device__ __forceinline__ T nbr_sum_par(uint32_t X, const T *u, const G2 &G, int par, int64_t &x) {
    const uint32_t m = X >> 1;
    const T *v = u + (par ? 0 : G.lay.ho) + m;
    const int64_t sy = G.sy, sz = G.sz;
    const int64_t xm = par - 1, xp = par, ym = par - ((sy + 1) >> 1), yp = par + ((sy - 1) >> 1);
    T s = (v[xm] + v[xp]) + (v[ym] + v[yp]);
    if (D == 3) {
        const int64_t zm = par - ((sz + 1) >> 1), zp = par + ((sz - 1) >> 1);
        s += v[zm] + v[zp];
    }
    x = (par ? G.lay.ho : 0) + m;  // the node's own slot
    return s;
}

template <int D, typename T>
__device__ __forceinline__ void smooth_at_par(uint32_t X, T *u, const T *Fs, const G2 &G, int par) {
    int64_t x;
    const T s = nbr_sum_par<D, T>(X, u, G, par, x);
    u[x] = fma(s, (T)G.inv_diag, Fs[x]);
}

// Fs of an interior row from its F
template <typename T>
__device__ __forceinline__ T scaled_rhs(T f, const G2 &G) {
    return (T)G.h2 * f * (T)G.inv_diag;
}

// interior residual (eq. Laph, with the reaction term c u)
template <int D, typename T>
__device__ __forceinline__ T residual_int(int64_t X, const T *u, const T *F, const G2 &G) {
    const T s = nbr_sum<D, T>(u, X, G);
    const int64_t x = pos(X, G.lay);
    return F[x] - ((T)G.diag * u[x] - s) * (T)G.ih2;
}

// Restriction (Sec. 2.1 eq. coarseFW, Sec. 3.3.2): FW if all 3^d fine
// neighbours belong to the coarse node's class family, else the FW-weight
// average over the family members.  FW weights are the integers 1, 2, 4
// (, 8) over 4^d; scaling by a power of two is exact.  The family of each
// coarse row is fixed by the classes, so it is computed once at set-up as a
// bit mask (family_mask); the cycle loads the mask and the members'
// residuals only (restrict_masked), all loads issued before any is used.
template <int D>
__device__ __forceinline__ bool restrict_nbr(const int ic[3], int k, const G2 &Gf, int64_t &Y) {
    const int ox = k % 3 - 1, oy = (k / 3) % 3 - 1, oz = (D == 3) ? k / 9 - 1 : 0;
    const int y0 = 2 * ic[0] + ox, y1 = 2 * ic[1] + oy, y2 = 2 * ic[2] + oz;
    Y = (int64_t)y0 + (int64_t)y1 * Gf.sy + (int64_t)y2 * Gf.sz;
    return y0 >= 0 && y0 <= Gf.N && y1 >= 0 && y1 <= Gf.N && (D == 2 || (y2 >= 0 && y2 <= Gf.N));
}

// the fine class bytes around coarse node ic (outside the grid: never in a
// family)
template <int D>
__device__ __forceinline__ void restrict_classes(const int ic[3], const uint8_t *clsf, const G2 &Gf,
                                                 uint8_t c[(D == 3) ? 27 : 9]) {
#pragma unroll
    for (int k = 0; k < ((D == 3) ? 27 : 9); ++k) {
        int64_t Y;
        c[k] = restrict_nbr<D>(ic, k, Gf, Y) ? clsf[Y] : (uint8_t)CL_BOXDIR;
    }
}

// reciprocals 1/w (correctly rounded) of the family weight sums 1..64
__device__ const double c_rcp64[65] = {
    0.0, 1.0 / 1, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8, 1.0 / 9, 1.0 / 10, 1.0 / 11,
    1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21,
    1.0 / 22, 1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29, 1.0 / 30, 1.0 / 31,
    1.0 / 32, 1.0 / 33, 1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39, 1.0 / 40, 1.0 / 41,
    1.0 / 42, 1.0 / 43, 1.0 / 44, 1.0 / 45, 1.0 / 46, 1.0 / 47, 1.0 / 48, 1.0 / 49, 1.0 / 50, 1.0 / 51,
    1.0 / 52, 1.0 / 53, 1.0 / 54, 1.0 / 55, 1.0 / 56, 1.0 / 57, 1.0 / 58, 1.0 / 59, 1.0 / 60, 1.0 / 61,
    1.0 / 62, 1.0 / 63, 1.0 / 64};
__device__ const float c_rcp32[65] = {
    0.0f, 1.0f / 1, 1.0f / 2, 1.0f / 3, 1.0f / 4, 1.0f / 5, 1.0f / 6, 1.0f / 7, 1.0f / 8, 1.0f / 9, 1.0f / 10,
    1.0f / 11, 1.0f / 12, 1.0f / 13, 1.0f / 14, 1.0f / 15, 1.0f / 16, 1.0f / 17, 1.0f / 18, 1.0f / 19,
    1.0f / 20, 1.0f / 21, 1.0f / 22, 1.0f / 23, 1.0f / 24, 1.0f / 25, 1.0f / 26, 1.0f / 27, 1.0f / 28,
    1.0f / 29, 1.0f / 30, 1.0f / 31, 1.0f / 32, 1.0f / 33, 1.0f / 34, 1.0f / 35, 1.0f / 36, 1.0f / 37,
    1.0f / 38, 1.0f / 39, 1.0f / 40, 1.0f / 41, 1.0f / 42, 1.0f / 43, 1.0f / 44, 1.0f / 45, 1.0f / 46,
    1.0f / 47, 1.0f / 48, 1.0f / 49, 1.0f / 50, 1.0f / 51, 1.0f / 52, 1.0f / 53, 1.0f / 54, 1.0f / 55,
    1.0f / 56, 1.0f / 57, 1.0f / 58, 1.0f / 59, 1.0f / 60, 1.0f / 61, 1.0f / 62, 1.0f / 63, 1.0f / 64};

// a / w for an integer weight sum 1 <= w <= 64 by Markstein's correction
// (P. W. Markstein, IBM J. Res. Dev. 34(1), 1990; the theorem in Muller et
// al., Handbook of Floating-Point Arithmetic, on correcting a quotient with
// one FMA): y = RN(1/w) from the table, q = RN(a y), the remainder
// r = a - q w is exact in one FMA, and RN(q + r y) is the correctly rounded
// a / w whenever y is the correctly rounded reciprocal, q lies within one
// ulp of a / w and nothing underflows.  A divide subroutine costs tens of
// FP64 instructions; this costs one multiply and two FMAs
// (bcmg_selftest_div_wsum checks it against true division).
template <typename T>
__device__ __forceinline__ T div_wsum(T a, int w) {
    const T y = sizeof(T) == 8 ? (T)c_rcp64[w] : (T)c_rcp32[w];
    const T q = a * y;
    const T r = fma(-q, (T)w, a);
    return fma(r, y, q);
}

// FW weight (1, 2, 4, 8) of fine neighbour k, and the bits of the
// neighbours with weight w
template <int D>
__host__ __device__ constexpr int fw_weight(int k) {
    return (k % 3 == 1 ? 2 : 1) * ((k / 3) % 3 == 1 ? 2 : 1) * ((D == 3 && k / 9 == 1) ? 2 : 1);
}

template <int D>
__host__ __device__ constexpr uint32_t fw_bits(int w) {
    uint32_t m = 0;
    for (int k = 0; k < ((D == 3) ? 27 : 9); ++k)
        if (fw_weight<D>(k) == w) m |= 1u << k;
    return m;
}

// The restriction's class family of a coarse node as a bit mask, fixed once
// the classes exist: bit k is set when fine neighbour k lies in the grid and
// in the family (interior node: interior; ghost: ghost or inactive)
template <int D>
__device__ __forceinline__ uint32_t family_mask(const int ic[3], bool interior, const uint8_t *clsf, const G2 &Gf) {
    uint8_t c[(D == 3) ? 27 : 9];
    restrict_classes<D>(ic, clsf, Gf, c);
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < ((D == 3) ? 27 : 9); ++k) {
        const bool fam = interior ? (c[k] == CL_INTERIOR) : (c[k] == CL_GHOST || c[k] == CL_INACTIVE);
        m |= fam ? (1u << k) : 0u;
    }
    return m;
}

// restrict_with from the family mask: the same terms in the same order (a
// non-member adds an exact zero), the weight sum from population counts
template <int D, typename T, bool CG = false>
__device__ __forceinline__ T restrict_masked(const int ic[3], uint32_t mask, const T *rf, const G2 &Gf) {
    constexpr int NT = (D == 3) ? 27 : 9;
    T v[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        const int ox = k % 3 - 1, oy = (k / 3) % 3 - 1, oz = (D == 3) ? k / 9 - 1 : 0;
        const int64_t Y = (int64_t)(2 * ic[0] + ox) + (int64_t)(2 * ic[1] + oy) * Gf.sy +
                          (int64_t)(2 * ic[2] + oz) * Gf.sz;
        v[k] = ((mask >> k) & 1u) ? ldv<CG>(rf + pos(Y, Gf.lay)) : T(0);
    }
    T fw = T(0);
#pragma unroll
    for (int k = 0; k < NT; ++k) fw = fma((T)fw_weight<D>(k), v[k], fw);
    if (mask == (1u << NT) - 1u) return fw * (D == 3 ? T(1.0 / 64.0) : T(1.0 / 16.0));
    const int wsum = __popc(mask & fw_bits<D>(1)) + 2 * __popc(mask & fw_bits<D>(2)) +
                     4 * __popc(mask & fw_bits<D>(4)) + 8 * __popc(mask & fw_bits<D>(8));
    return wsum > 0 ? div_wsum<T>(fw, wsum) : T(0);
}

// multilinear prolongation at fine node iy (Sec. 2.1, 3.2, 3.3.2): the 2^k
// coarse neighbours (k = number of odd coordinates) all weigh 2^-k, so their
// sum is scaled once; the corner loads are predicated, not branched
template <int D, typename T, bool CG = false>
__device__ __forceinline__ T prolong_at(const int iy[3], const T *ec, const G2 &Gc) {
    const int t0 = iy[0] & 1, t1 = iy[1] & 1, t2 = (D == 3) ? (iy[2] & 1) : 0;
    const int64_t C0 = (int64_t)(iy[0] >> 1) + (int64_t)(iy[1] >> 1) * Gc.sy +
                       (D == 3 ? (int64_t)(iy[2] >> 1) * Gc.sz : 0);
    constexpr int NC = (D == 3) ? 8 : 4;
    T c[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int b0 = k & 1, b1 = (k >> 1) & 1, b2 = (k >> 2) & 1;
        const bool p = b0 <= t0 && b1 <= t1 && b2 <= t2;
        c[k] = p ? ldv<CG>(ec + pos(C0 + b0 + b1 * Gc.sy + b2 * Gc.sz, Gc.lay)) : T(0);
    }
    T v = c[0];
    if (t0) v += c[1];
    if (t1) {
        v += c[2];
        if (t0) v += c[3];
    }
    if (D == 3 && t2) {
        v += c[4];
        if (t0) v += c[5];
        if (t1) {
            v += c[6];
            if (t0) v += c[7];
        }
    }
    const int k = t0 + t1 + t2;
    const T scale = k == 0 ? T(1) : k == 1 ? T(0.5) : k == 2 ? T(0.25) : T(0.125);
    return v * scale;
}

// the map of the first kEllFirst terms of band node b (read before the
// dependency wait)
constexpr int kEllFirst = 16;

template <typename T>
struct EllRound {
    int c;
    uint32_t g[kEllFirst];
    T w[kEllFirst];
};

template <typename T>
__device__ __forceinline__ void ell_first(int64_t b, const uint8_t *ecnt, const uint32_t *eg, const double *ew,
                                          int64_t nb, EllRound<T> &R) {
    R.c = ecnt[b];
#pragma unroll
    for (int j = 0; j < kEllFirst; ++j) {
        const bool p = j < R.c;
        R.g[j] = p ? eg[(int64_t)j * nb + b] : 0u;
        R.w[j] = p ? (T)ew[(int64_t)j * nb + b] : T(0);
    }
}

// band value: the expanded extension (ELL terms of band node b, term-major)
// with the map of its first terms already loaded, the rest in rounds of
// eight with predicated loads so that their gathers overlap
template <typename T>
__device__ __forceinline__ T extend_from(int64_t b, const EllRound<T> &R, const uint32_t *eg, const double *ew,
                                         int64_t nb, const T *a, Lay ly) {
    T v = T(0);
    {
        T x[kEllFirst];
#pragma unroll
        for (int j = 0; j < kEllFirst; ++j) x[j] = j < R.c ? a[pos(R.g[j], ly)] : T(0);
#pragma unroll
        for (int j = 0; j < kEllFirst; ++j)
            if (j < R.c) v = fma(R.w[j], x[j], v);
    }
    for (int k0 = kEllFirst; k0 < R.c; k0 += 8) {
        T w[8], x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool p = k0 + j < R.c;
            const int64_t e = (int64_t)(k0 + j) * nb + b;
            w[j] = p ? (T)ew[e] : T(0);
            x[j] = p ? a[pos(eg[e], ly)] : T(0);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (k0 + j < R.c) v = fma(w[j], x[j], v);
    }
    return v;
}

// ------------------------------------------------------------ norms
// the block's norm partials (sum r^2, max|r|) of one row class, reduced in
// a fixed order (warp shuffles, then the block's warps); every thread calls it
// max |r| is carried as the bit pattern of a non-negative double: integer
// order is numeric order there, so the maxima run on the integer pipe
// (FP64 issue slots are the scarce resource)
__device__ __forceinline__ long long abs_bits(double v) { return __double_as_longlong(v) & 0x7fffffffffffffffLL; }

__device__ __forceinline__ void block_partials(double s2, long long mxb, double *part, int64_t slot, bool interior) {
    __shared__ double sh[kT / 32];
    __shared__ long long shm[kT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        mxb = max(mxb, __shfl_down_sync(0xffffffffu, mxb, o));
    }
    if (lane == 0) {
        sh[warp] = s2;
        shm[warp] = mxb;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        s2 = lane < nw ? sh[lane] : 0.0;
        mxb = lane < nw ? shm[lane] : 0LL;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s2 += __shfl_down_sync(0xffffffffu, s2, o);
            mxb = max(mxb, __shfl_down_sync(0xffffffffu, mxb, o));
        }
        if (lane == 0) {
            const double mx = __longlong_as_double(mxb);
            double *p = part + slot * 4;
            p[0] = interior ? s2 : 0.0;
            p[1] = interior ? 0.0 : s2;
            p[2] = interior ? mx : 0.0;
            p[3] = interior ? 0.0 : mx;
        }
    }
}

// norms of the residual (interior, ghost) -> sqrt(a^2 + b^2), rounded step by step
__device__ __forceinline__ double resid_norm(const double *nout) {
    return __dsqrt_rn(__dadd_rn(__dmul_rn(nout[0], nout[0]), __dmul_rn(nout[1], nout[1])));
}

__device__ __forceinline__ bool finite_d(double x) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) < 0x7ff0000000000000LL;
}

}  // namespace
}  // namespace bcmg
