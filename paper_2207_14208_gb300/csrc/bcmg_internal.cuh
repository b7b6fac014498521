// Internal declarations of the GB300 BCMG library (not part of the C ABI).
//
// Data layout in HBM, per level l (N_l = N >> l cells, n_l = N_l + 1 nodes per
// axis; node X = i + n j + n^2 k; cls dense x-fastest, the value arrays u, F,
// Fs, r parity-split, see split_ho below):
//   cls  uint8 node class (INACTIVE / INTERIOR / GHOST / BOXDIR)
//   u    FP64 solution (level 0: internal copy) or correction e (l > 0)
//   F    FP64 right-hand side: f on interior rows, g on ghost rows (level 0),
//        restricted residuals on coarse levels
//   r    FP64 residual (interior, ghost, then extended into the band)
// Work lists (compacted once at set-up):
//   ilist interior node indices, red nodes ((i + j + k) even) first, then
//        black, each colour in increasing index order; one thread per node
//   ghost list: index, direction/degree code, xi per axis (SoA), Delta tau
//   band list: index, up to d upwind sources (band position or ghost index)
//        with normalised weights (SoA)
//   coarsest level: active list and the dense inverse of its system
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "bcmg.h"

namespace bcmg {

enum : uint8_t { CL_INACTIVE = 0, CL_INTERIOR = 1, CL_GHOST = 2, CL_BOXDIR = 3 };

constexpr int kMaxCoarse = 4096;   // largest coarsest system inverted densely
#ifndef BCMG_TAIL_NODES
#define BCMG_TAIL_NODES 8192
#endif
constexpr int kTailNodes = BCMG_TAIL_NODES;  // coarse levels up to this many interior +
                                             // ghost + band nodes run in the cluster tail
constexpr int kTailCoarse = 1024;  // largest coarsest system the tail inverts
constexpr int32_t kNoRef = INT32_MIN;

// Level arrays of values (u, F, Fs, r and their FP32 copies) are stored
// parity-split: node X (linear index i + n j + n^2 k) lives at position
// (X >> 1) + (X & 1) ho, the even-index nodes first, the odd-index nodes
// from offset ho on.  Every smoothed level has an odd n = N + 1, and then
// the parity of X is the red-black colour (i + j + k) mod 2, so each colour
// is one contiguous half: a sweep reads the other colour's half and writes
// its own densely.  ho is ceil(nn / 2) rounded up to 32 entries.
__host__ __device__ __forceinline__ int64_t split_ho(int64_t nn) { return ((nn + 1) / 2 + 31) / 32 * 32; }
__host__ __device__ __forceinline__ int64_t split_len(int64_t nn) { return split_ho(nn) + nn / 2; }
// A level's layout: position of node X = (X >> s) + ((X & m) ? ho : 0):
// s = m = 1 and ho = split_ho(nn) for the parity-split layout (the grid
// levels), s = m = ho = 0 for the dense one (the small levels of the cluster
// tail, where the split layout only lengthens latency-bound gathers).  Node
// indices and positions are below 2^32 (checked at creation); 32-bit
// arithmetic keeps the address chains short.
struct Lay {
    uint32_t s = 1, m = 1, ho = 0;
};
__host__ __device__ __forceinline__ uint32_t pos(int64_t X, const Lay &y) {
    const uint32_t x = (uint32_t)X;
    return (x >> y.s) + ((x & y.m) ? y.ho : 0u);
}

struct Level {
    int d = 0, N = 0, n = 0;
    int64_t nn = 0;
    Lay lay;  // layout of the value arrays (parity-split unless a tail level)
    int64_t st[3] = {0, 0, 0};
    double h = 0.0;
    double lo = -1.0;  // coordinate of node 0 on every axis (x_i = lo + i h)
    double react = 0.0;  // reaction coefficient c of c u - Lap u = f
    uint8_t *cls = nullptr;
    int64_t nint = 0, nbox = 0, ng = 0, nb = 0, nclamp = 0, nfall = 0, nact = 0;
    int64_t nred = 0;            // red interior nodes (head of ilist)
    int64_t nbn = 0;             // black interior nodes next to a ghost or box-edge node
    uint32_t *ilist = nullptr;  // nint interior node indices, red then black (each part sorted)
    uint32_t *bnear = nullptr;  // the nbn black nodes next to a ghost or box-edge node, sorted
    uint32_t *bmask = nullptr;  // bit j set: black entry ilist[nred + j] is in bnear
    // GS-LEX order only: interior nodes grouped by hyperplane p = i + j (+ k),
    // hyperplane p at hlist[hoff[p] .. hoff[p + 1])
    uint32_t *hlist = nullptr;
    std::vector<int64_t> hoff;
    // ghosts (SoA)
    uint32_t *gidx = nullptr;
    uint16_t *gcode = nullptr;  // bit a: s_a = -1; bits 3+2a..4+2a: degree q_a
    double *gxi = nullptr;      // 3 * ng, axis-major
    double *gdt = nullptr;
    double *geta = nullptr;
    double *gn = nullptr;  // 3 * ng, axis-major
    double *gQ = nullptr;  // ng * d, point-major (x, y[, z])
    // interpolation weights of B at each ghost: 3^d terms (o2 * 3 + o1) * 3
    // + o0, term-major (gw[term * ng + g]); FP32 copy for the mixed cycle
    double *gw = nullptr;
    float *gw32 = nullptr;
    // restriction family of each coarse row (interior rows, then ghosts):
    // bit k for fine neighbour k (levels >= 1)
    uint32_t *fmask = nullptr;
    // band (SoA)
    uint32_t *bidx = nullptr;
    int32_t *bref = nullptr;  // 3 * nb, axis-major: >= 0 band position,
                              // < 0 -(ghost node index) - 1, kNoRef none
    double *bw = nullptr;     // 3 * nb, axis-major, normalised weights
    // the K extension sweeps from zero are a fixed linear map from ghost
    // values to band values: per band node up to kExtCap (ghost node,
    // weight) terms, ELL layout (term-major); null ecnt = sweep by sweep
    uint8_t *ecnt = nullptr;  // nb
    int ell_max = 0;          // longest row
    uint32_t *eg = nullptr;   // kExtCap * nb
    double *ew = nullptr;     // kExtCap * nb
    // boxdir list (finest level only)
    uint32_t *boxidx = nullptr;
    // arrays
    double *u = nullptr, *F = nullptr, *r = nullptr;
    double *Fs = nullptr;  // h^2 F / (2d + c h^2) on the interior rows (smoothing)
    double *gtmp = nullptr;  // ng
    double *bbuf = nullptr;  // 2 * nb
    // FP32 arrays of the mixed-precision inner cycle (correction equation)
    float *u32 = nullptr, *F32 = nullptr, *r32 = nullptr, *gtmp32 = nullptr, *bbuf32 = nullptr;
    float *Fs32 = nullptr;
    // coarsest
    uint32_t *act = nullptr;
    double *Ainv = nullptr;
    double *crhs = nullptr;
    // set-up only: phi of this level (finest: caller's array)
    const double *phi = nullptr;
};

// device-side state of a solve run as one graph (WHILE conditional node)
struct SolveState {
    double rtol;     // in: stop when ||r|| / ||r0|| <= rtol
    int max_cycles;  // in
    int cycles;      // out: cycles done
    double r0, rel;  // out: initial residual norm, final relative residual
    int status;      // out: BCMG_OK or BCMG_ENONFINITE
};

constexpr uint32_t kHandleMagic = 0x474d4342u;  // set while a handle is live

struct Arena {  // bump allocation inside one zero-filled device chunk
    char *base = nullptr;
    size_t used = 0, cap = 0;
};

struct Handle {
    uint32_t magic = kHandleMagic;
    int d = 0;
    int64_t N = 0;
    bcmg_opts o{};
    cudaStream_t user = nullptr;  // caller's stream
    cudaStream_t st = nullptr;    // library stream (graph capture, all work)
    cudaStream_t st2 = nullptr;   // side stream of creation (coarsest inverse)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<Level> L;
    double *u0 = nullptr;        // finest-level working copy of u
    double *npart = nullptr;     // norm partials
    unsigned *ncount = nullptr;  // blocks of the ghost residual done (zero between launches)
    int *sing_host = nullptr;    // coarsest-system singular flag (pinned block; read after creation's sync)
    double *nout = nullptr;      // 4 norms (device)
    double *nhost = nullptr;     // pinned copy of the 4 norms
    cudaGraphExec_t vgraph = nullptr;
    cudaGraphExec_t ngraph = nullptr;  // V-cycle followed by norms
    // whole solve on the device: norms, then WHILE (cycle, norms, check)
    cudaGraphExec_t sgraph = nullptr;
    bool sgraph_failed = false;  // graph with a conditional node unavailable
    int64_t sgraph_prefix = 0, sgraph_body = 0;  // kernels before / per iteration
    SolveState *sdev = nullptr, *shost = nullptr;
    SolveState *shost_dev = nullptr;  // device address of shost (null: copies instead)
    int64_t vgraph_kernels = 0, ngraph_kernels = 0;
    // coarse end of the V-cycle on one thread-block cluster: first level (-1:
    // none), cluster size
    // and the per-level tables of the FP64 and FP32 cycles
    int tail_start = -1, tail_cluster = 0;
    void *tail64 = nullptr, *tail32 = nullptr;
    void *tail_ops = nullptr;  // (kind, level) schedule of the tail
    int tail_nops = 0;
    int nsm = 152;  // SMs of the device (block sizes of the FP64 kernels)
    int pers_blocks = 0;  // resident blocks of the persistent FP32 sweep (0: not yet queried)
    int dev = 0;    // the device the handle was created on
    bool capturing = false;
    int64_t captured = 0;
    std::vector<std::pair<void *, size_t>> allocs;
    int64_t dev_bytes = 0;      // device memory the handle holds
    double lo = -1.0;           // domain box [lo, lo + N h0]^d
    double h0 = 0.0;            // finest grid spacing
    // caller-supplied workspace: every device array of the handle (set-up
    // scratch included) is carved from it; no pool allocation
    char *ws_base = nullptr;
    size_t ws_cap = 0, ws_used = 0;
    int64_t alloc_total = 0;    // bytes drawn during creation (perm + scratch)
    double *stage[3] = {nullptr, nullptr, nullptr};  // split scratch of the stage operators
    Arena arena_perm, arena_temp;
    std::vector<std::pair<void *, size_t>> temps;  // set-up scratch, freed when creation ends
    // profiling of the finest-level sweeps (opts.profile)
    std::vector<cudaEvent_t> pev;
    int pev_next = 0, pev_pairs = 0;
    double prof_ms = 0.0;
    int64_t prof_n = 0;
};

// record a timing event of the finest-level sweep profile (no-op otherwise)
void profile_mark(Handle &H, const Level &L);

// ---- error handling -------------------------------------------------
struct Error {
    int code;
    std::string msg;
};
void check_cuda(cudaError_t e, const char *what);
// device array of the handle; temp: freed when creation ends; zero: the
// array must start zero-filled (small arrays always are)
void *dalloc(Handle &H, size_t bytes, bool temp = false, bool zero = true);
void count_launch(Handle &H);
int64_t launches_total();
void add_launches(int64_t n);
int report(int code, const std::string &msg);  // sets the thread's last error
int selftest_div_wsum(int fp32, const double *a_host, int64_t n, double *out_host, std::string *msg);

// ---- set-up (setup.cu) -------------------------------------------------
void setup_hierarchy(Handle &H, const double *phi0);
double dtau_of(int d, int bc, int mode, double cst, double theta);
bool ext_ell_ok(int d, int K);
constexpr int kExtCap = 32;  // terms per band node of the expanded extension

// ---- cycle kernels (cycle.cu); T = double (FP64) or float (inner cycles of
// the mixed-precision refinement) ----------------------------------------
// Fs: the level's scaled right-hand side (the cycle), or null (a caller's F)
template <typename T> void smooth(Handle &H, Level &L, T *u, const T *F, int nsteps, const T *Fs = nullptr);
// after_rb: u comes straight from a red-black smoothing step of this level
// (black rows whose neighbours are all interior then hold a zero residual)
template <typename T> void residual(Handle &H, Level &L, const T *u, const T *F, T *r, bool after_rb = false);
template <typename T> void extend(Handle &H, Level &L, T *a);
// early_ok: the fine level's residual (and band extension) are the launches
// right before
template <typename T>
// Fsc: where the coarse interior rows' scaled right-hand side goes (or null)
void restrict_to(Handle &H, Level &Lf, Level &Lc, const T *rf, T *Fc, T *uc_zero, bool early_ok = false,
                 T *Fsc = nullptr);
// early_ok: the coarse correction's extension is the launch right before
template <typename T> void prolong(Handle &H, Level &Lf, Level &Lc, const T *ec, T *uf, bool early_ok = false);
template <typename T> void coarsest_correct(Handle &H, Level &L, T *u, const T *F);
// finest-level residual r = F - A u and its four norms (out4, device);
// ctl 1 / 2 also enqueue the solve's start / per-cycle check on cond
void residual_norms(Handle &H, const double *u, double *out4, int ctl = 0, unsigned long long cond = 0,
                    bool after_rb = false);
int64_t norm_parts(const Level &L);  // block partials residual_norms writes
// ghost weights of every level; the levels of the cluster tail and their tables
void setup_cycle(Handle &H);
// device-side solve control: initial and per-cycle convergence checks that
// set the WHILE condition of the solve graph
void solve_init_enqueue(Handle &H, unsigned long long cond);
void solve_check_enqueue(Handle &H, unsigned long long cond);
void vcycle_enqueue(Handle &H, int l, double *u);
// summed device time (ms) of nsweeps back-to-back finest-level colour sweeps
double time_sweeps(Handle &H, int nsweeps);
double time_sweeps_bf16(Handle &H, int nsweeps);
// batched solves (batch.cu): can these hierarchies advance together (same
// dimension, precision, device, red-black V(nu1, nu2) cycles, expanded
// extensions)?  Then solve all of them from their working copies u0, ordered
// on st; per-hierarchy cycles, relative residuals and statuses into the host
// arrays; returns the kernels launched.
bool batch_eligible(const std::vector<Handle *> &hs);
// launch shape of the batched kernels for the following batched solves
// instead of the autotuner's (block <= 0: back to the autotuner)
void batch_shape_override(int block, int items, int64_t tail_rows);
// the launch shape the last batched solve of the process used (block 0: none yet)
void batch_last_shape(int *block, int *items, int64_t *tail_rows);
// every handle's u between the caller's arrays and the working copies (in:
// interior, ghost and eliminated box nodes; out: interior and ghost nodes),
// one launch on st
void batch_copy_active(const std::vector<Handle *> &hs, double *const *u_devs, cudaStream_t st, bool in);
int64_t batch_solve(const std::vector<Handle *> &hs, cudaStream_t st, double rtol, int max_cycles, int *cycles,
                    double *rels, int *statuses, bool fixed = false);
// one refinement step: F32 = r (finest), FP32 V-cycle on the correction,
// u += correction; r must hold the FP64 residual of u
void mixed_step_enqueue(Handle &H, double *u);
// in: the caller's dense u (interior, ghost and eliminated box nodes) into
// the finest working copy (parity-split); otherwise the working copy's
// interior and ghost nodes back into the caller's dense array
void copy_active(Handle &H, const double *src, double *dst, bool in);
// whole level arrays between the caller's dense layout and the split one
void dense_to_split(Handle &H, const Level &L, const double *dense, double *split);
void split_to_dense(Handle &H, const Level &L, const double *split, double *dense);
void scatter_ghost_values(Handle &H, Level &L, const double *g, double *F);
void set_interior_rhs(Handle &H, Level &L, const double *f, double *F);

}  // namespace bcmg
