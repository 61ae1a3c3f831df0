// abi.cu -- the C ABI of libafqmc.so (include/afqmc.h): contexts, walkers and
// the orchestration of one slice of the PQMC sweep (Sec. II.B-II.D, III).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"
#include "sepwrap.cuh"

namespace afq {
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches += n; }

// A kernel attribute set by cudaFuncSetAttribute belongs to the kernel on the current device, so
// the cache is keyed by (device, kernel, attribute) and guarded by a mutex; the attribute is set
// again only when a larger value is asked for on that device.
cudaError_t ensure_func_attr(const void* fn, cudaFuncAttribute attr, int value) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, int>, int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(dev, fn, (int)attr);
    auto it = done.find(key);
    if (it != done.end() && it->second >= value) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, attr, value);
    if (e == cudaSuccess) done[key] = value;
    return e;
}
}  // namespace afq

using namespace afq;

namespace {

struct Lattice {
    int L = 0, N = 0;
    long ld = 0;
    double* E64 = nullptr;
    double* Einv64 = nullptr;
    void* Eb = nullptr;
    void* Einvb = nullptr;
    double* Ex64 = nullptr;   // L x L: exp(-dtau K) = Ex (x) Ex for the periodic square lattice
    double* Exi64 = nullptr;  // L x L: exp(+dtau K) = Exi (x) Exi
};

// A group of walkers with the same lattice and particle numbers.  Every per-walker buffer holds
// nwk back-to-back copies laid out [walker][spin][...], so the walker and spin indices of a
// launch merge into one batch index with a uniform stride.
struct Walker {
    int nwk = 1;             // walkers in the group
    std::vector<int> gid;    // their indices in the context (also their Philox key)
    int* gid_d = nullptr;
    int L = 0, N = 0;
    long ld = 0;
    int ns[2] = {0, 0};
    int nsm = 0;             // max(ns[0], ns[1])
    int nst = 0;             // stack entries (M / stab_every + 1)
    int pos = 0, last_dir = -1;
    bool need_recompute = false;
    uint64_t visit = 0;
    Lattice* lat = nullptr;
    void* G = nullptr;       // [nwk][2][N][ld] bulk
    void* Tbuf = nullptr;    // [nwk][2][N][ld] bulk (wrap temporary)
    int8_t* x = nullptr;     // [nwk][M][N]
    double* u = nullptr;     // [nwk][2N] uniforms
    void* dvec = nullptr;    // bulk [nwk][2][N] d, then [nwk][2][N] dinv
    double* d64 = nullptr;   // FP64 [2][N] d, [2][N] dinv (one walker at a time)
    uint8_t* dec = nullptr;  // [nwk][2N]
    double* ratio = nullptr; // [nwk][2N]
    int* stats = nullptr;    // [nwk][8]
    double* maxr = nullptr;  // [nwk]
    double* sign = nullptr;  // [nwk]
    uint8_t* replay = nullptr;
    void* colbuf = nullptr;
    void* rowbuf = nullptr;
    GridBar* bar = nullptr;
    int* err = nullptr;
    // window buffers, double-buffered by window parity (the flush of window w overlaps the
    // decisions of window w + 1), and the corrected snapshots of the next window's block
    int* wm[2] = {nullptr, nullptr};
    int* widx[2] = {nullptr, nullptr};
    double* wdtot[2] = {nullptr, nullptr};
    void* Wm[2] = {nullptr, nullptr};
    void* Wx[2] = {nullptr, nullptr};
    void* X[2] = {nullptr, nullptr};
    void* Y[2] = {nullptr, nullptr};
    void* snap[2] = {nullptr, nullptr};
    cudaStream_t sf = nullptr;  // flush stream
    cudaStream_t sp = nullptr;  // propagation stream: the next recompute's factor, one slice behind the sweep
    cudaEvent_t ev_wrap = nullptr, ev_prop = nullptr;  // after each slice's wrap; after the last propagation
    int prop_pos = -1, prop_dir = 0;  // Ucur holds the factor at prop_pos (direction prop_dir) after ev_prop
    int pend_slice = 0;               // forward slice whose propagation waits for the next slice's wrap
    // FP32 bulk, G form: slices of propagation in the current factor since its last
    // re-orthonormalisation (reset when the sweep turns), and the direction it counts for
    int orth_since = 0, orth_dir = 0;
    cudaStream_t sm = nullptr;  // the group's main stream (forked from the caller's stream)
    cudaEvent_t ev_chain[2] = {nullptr, nullptr}, ev_prod[2] = {nullptr, nullptr}, ev_done = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_rc = nullptr;  // after a recompute's last read of the propagated factor (deferred LU)
    unsigned long long* visit_d = nullptr;  // device visit counter (keys the uniforms)
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        long long launches = 0;
    };
    std::map<long long, Graph> graphs;  // captured slices by (slice, dir, mode, k, nb)
    double* URs = nullptr;   // [nwk][2][nst][N x nsm]: right factors at every recompute point
    double* ULs = nullptr;   // [nwk][2][nst][nsm x N]: left factors
    double* Ucur = nullptr;  // [nwk][2][N x nsm]: the factors being propagated
    double* Utmp = nullptr;  // N x nsm: propagation scratch (per-slice path)
    double* Ut2 = nullptr;   // [nwk][2][N x nsm]: transposed left factors for the LU
    double* Ob = nullptr;    // [nwk][2][nsm x nsm]: U_L U_R, then its LU
    double* Z = nullptr;     // [nwk][2][nsm x N]: (U_L U_R)^{-1} U_L
    double* Gnew = nullptr;  // [nwk][2][N][ld]: the recomputed G
    int* perm2 = nullptr;    // [nwk][2][maxr]: pivot rows
    int8_t* flag2 = nullptr; // [nwk][2][maxr]: pivoted-row flags
    int* visited = nullptr;  // [nwk][maxr]: permutation-parity scratch
    double* acc2 = nullptr;  // [nwk][2]
    // the recompute's two FP64 products on the tensor cores (digit splitting, ozaki.cu)
    bool oz_Z = false, oz_G = false;  // U_L U_R, and U_R Z
    void* ozw = nullptr;              // digit planes, both products (the spin groups run in turn)
    double* ozs = nullptr;            // row / column scales
    // T form (afqmc_set_form): U_R [nwk][2][N x nsm], U_L [nwk][2][nsm x N], T [nwk][2][nsm x nsm] in
    // the bulk precision; the window gathers U_L[:, I] (nsm x NW) and U_R[I, :] (NW x nsm), the
    // products V = T U_L[:, I], Y = U_R[I, :] T and Y' = W Y, the rows U_R[J, :] T of the next
    // window (NW x nsm); an FP64 identity (nsm x nsm): T = 1 after every recompute
    void *TUR = nullptr, *TUL = nullptr, *TT = nullptr;
    void *ULI = nullptr, *URI = nullptr, *Vt = nullptr, *Yt = nullptr, *Ypt = nullptr, *Pt = nullptr;
    double* Ieye = nullptr;
    // G form with FP32 bulk and digit-split products: (U_L U_R)^{-1} explicitly (nsm x nsm per
    // matrix), so that Z = O^{-1} U_L runs on the tensor cores instead of an N-column solve
    double* Oinv = nullptr;
    bool gvalid = true;  // the bulk G buffer holds the current G (the T form forms it on request)
    // constrained-path AFQMC (afqmc_cp_*): per walker [sum ln N_i, sum ln |r_up r_dn|, removed, kinetic
    // ln ratio], the tracked ln |det U_L U_R| (both spins), per matrix ln |det|, per walker the sign,
    // and the walkers' ln weights (host)
    double *cpl = nullptr, *cpdet = nullptr, *cpla = nullptr, *cpsg = nullptr, *cpsref = nullptr;
    double* cptmp = nullptr;  // population control: [nwk][2 N n_s + 2 n_s^2 + 2] gather scratch
    std::vector<double> cp_logw;
    bool cp = false;
    std::vector<void*> allocs;
    long gstride() const { return 2L * N * ld; }
    int rows_max() const { return N > nsm ? N : nsm; }
    long fsz() const { return (long)N * nsm; }                  // one factor
    long st_s() const { return (long)nst * fsz(); }             // spin stride in a stack
    long st_w() const { return 2 * st_s(); }                    // walker stride in a stack
    double* stackR(int j) const { return URs + (size_t)j * fsz(); }
    double* stackL(int j) const { return ULs + (size_t)j * fsz(); }
};

}  // namespace

struct Prof {
    bool on = false;
    double ms[AFQMC_NPHASE] = {};
    int64_t intervals[AFQMC_NPHASE] = {};
    int64_t launches[AFQMC_NPHASE] = {};
    std::vector<cudaEvent_t> pool;
    struct Pend {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Pend> pending;
};

struct afqmc_ctx {
    Prof prof;
    afqmc_params p;
    double lam = 0.0, c[2] = {0.0, 0.0};
    int sticky = 0;
    int nsm = 0;
    bool graphs = false;  // replay captured slices (afqmc_set_graphs)
    int wrap_mode = -1;     // AFQMC_WRAP_* set by afqmc_set_wrap; -1: separable where the lattice fits
    int form = AFQMC_FORM_G;  // walker representation (afqmc_set_form, before afqmc_init_walkers)
    int sep_tile = 0;       // tile width of the separable passes (afqmc_set_wrap_tile; 0: the default)
    std::vector<Lattice*> lats;
    std::vector<Walker*> w;                        // walker groups
    std::vector<std::pair<int, int>> wmap;         // context walker -> (group, member)
    std::vector<size_t> roff;                      // context walker -> offset of its 2N replay bytes
    std::vector<void*> allocs;
    cudaStream_t last = nullptr;
};

#define CK(call)                                        \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return fail(ctx, e_);    \
    } while (0)

static int fail(afqmc_ctx* ctx, cudaError_t e) {
    int code = (e == cudaErrorMemoryAllocation) ? AFQMC_ERR_OOM : AFQMC_ERR_CUDA;
    if (ctx && ctx->sticky == 0) ctx->sticky = code;
    return code;
}

template <typename P>
static cudaError_t dalloc(std::vector<void*>& list, P** out, size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) return e;
    list.push_back(p);
    *out = (P*)p;
    return cudaSuccess;
}

static size_t esize(const afqmc_ctx* ctx) { return ctx->p.precision == AFQMC_PREC_FP64 ? 8 : 4; }

// ---------------------------------------------------------------------------
// small kernels local to the ABI layer
// ---------------------------------------------------------------------------
// B[b] = A[b]^T (A[b]: rows x cols) for the batch b = blockIdx.y, A[b] at A + b sa, B[b] at B + b sb
__global__ void transpose_kernel(const double* A, int rows, int cols, double* B, long sa, long sb) {
    A += blockIdx.y * sa;
    B += blockIdx.y * sb;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)rows * cols; e += (long)gridDim.x * blockDim.x) {
        int r = (int)(e / cols), c = (int)(e % cols);
        B[(long)c * rows + r] = A[e];
    }
}

__global__ void fields_kernel(uint64_t seed, uint64_t walker, long count, int8_t* x) {
    long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count) x[j] = philox_uniform(seed, walker, ~0ULL, (uint64_t)j) < 0.5 ? 1 : -1;
}

__global__ void set_double_kernel(double* p, double v, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// One thread waits for a flag that nothing sets, bounded by limit_ns of %globaltimer, then
// records DEV_TIMEOUT and returns: the path every bounded wait of the library takes on expiry.
__global__ void debug_wait_kernel(const unsigned int* flag, unsigned long long limit_ns, int* err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (*((volatile const unsigned int*)flag) != 0u) return;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
            set_err(err, DEV_TIMEOUT);
            return;
        }
        __nanosleep(1000);
    }
}

__global__ void debug_uniforms_kernel(uint64_t seed, uint64_t walker, uint64_t visit, int count, double* out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count) out[j] = philox_uniform(seed, walker, visit, (uint64_t)j);
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static int check_ctx(afqmc_ctx* ctx) {
    if (!ctx) return AFQMC_ERR_ARG;
    if (ctx->sticky) return ctx->sticky;
    return 0;
}

static cudaEvent_t prof_event(afqmc_ctx* ctx) {
    if (!ctx->prof.pool.empty()) {
        cudaEvent_t e = ctx->prof.pool.back();
        ctx->prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one phase with CUDA events on the launching stream (when profiling is on).
struct PhaseScope {
    afqmc_ctx* ctx;
    int ph;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    long long l0;
    PhaseScope(afqmc_ctx* c, int phase, cudaStream_t s) : ctx(c), ph(phase), st(s), l0(g_launches.load()) {
        if (ctx->prof.on) {
            a = prof_event(ctx);
            cudaEventRecord(a, st);
        }
    }
    ~PhaseScope() {
        if (!ctx->prof.on || !a) return;
        cudaEvent_t b = prof_event(ctx);
        cudaEventRecord(b, st);
        ctx->prof.pending.push_back({ph, a, b});
        ctx->prof.launches[ph] += g_launches.load() - l0;
    }
};

static int read_dev_err(afqmc_ctx* ctx, Walker* w) {
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, w->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(ctx, e);
    if (h == DEV_TIMEOUT) ctx->sticky = AFQMC_ERR_TIMEOUT;
    else if (h == DEV_NUMERIC) ctx->sticky = AFQMC_ERR_NUMERIC;
    else if (h != 0) ctx->sticky = AFQMC_ERR_CUDA;
    return ctx->sticky;
}

// E = exp(-dtau K), E^{-1} and the one-dimensional factor Ex of the L x L lattice, in FP64 and
// in the bulk precision.  Device buffers go to ctx->allocs (freed by afqmc_destroy).
static cudaError_t fill_lattice(afqmc_ctx* ctx, Lattice* l, cudaStream_t st) {
    const int L = l->L;
    const size_t n2 = (size_t)l->N * l->ld;
    cudaError_t e;
    if ((e = dalloc(ctx->allocs, &l->E64, n2 * 8)) != cudaSuccess) return e;
    if ((e = dalloc(ctx->allocs, &l->Einv64, n2 * 8)) != cudaSuccess) return e;
    if ((e = dalloc(ctx->allocs, (char**)&l->Eb, n2 * esize(ctx))) != cudaSuccess) return e;
    if ((e = dalloc(ctx->allocs, (char**)&l->Einvb, n2 * esize(ctx))) != cudaSuccess) return e;
    if ((e = dalloc(ctx->allocs, &l->Ex64, (size_t)L * L * 8)) != cudaSuccess) return e;
    if ((e = dalloc(ctx->allocs, &l->Exi64, (size_t)L * L * 8)) != cudaSuccess) return e;
    if ((e = launch_expK1d(st, L, ctx->p.t, ctx->p.dtau, l->Ex64)) != cudaSuccess) return e;
    if ((e = launch_expK1d(st, L, ctx->p.t, -ctx->p.dtau, l->Exi64)) != cudaSuccess) return e;
    if ((e = launch_expK(st, L, ctx->p.t, ctx->p.dtau, l->E64, l->ld)) != cudaSuccess) return e;
    if ((e = launch_expK(st, L, ctx->p.t, -ctx->p.dtau, l->Einv64, l->ld)) != cudaSuccess) return e;
    if (ctx->p.precision == AFQMC_PREC_FP64) {
        if ((e = launch_cast<double>(st, l->E64, l->ld, (double*)l->Eb, l->ld, l->N, l->N)) != cudaSuccess) return e;
        return launch_cast<double>(st, l->Einv64, l->ld, (double*)l->Einvb, l->ld, l->N, l->N);
    }
    if ((e = launch_cast<float>(st, l->E64, l->ld, (float*)l->Eb, l->ld, l->N, l->N)) != cudaSuccess) return e;
    return launch_cast<float>(st, l->Einv64, l->ld, (float*)l->Einvb, l->ld, l->N, l->N);
}

static Lattice* get_lattice(afqmc_ctx* ctx, int L, cudaStream_t st, cudaError_t* err) {
    for (auto* l : ctx->lats)
        if (l->L == L) return l;
    Lattice* l = new Lattice();
    l->L = L;
    l->N = L * L;
    l->ld = ((l->N + 31) / 32) * 32;
    if ((*err = fill_lattice(ctx, l, st)) != cudaSuccess) {
        delete l;
        return nullptr;
    }
    ctx->lats.push_back(l);
    return l;
}

static cudaError_t prop_right(afqmc_ctx* ctx, Walker* w, cudaStream_t st, int j, int s, int ell, double* U,
                              double* tmp);
static cudaError_t prop_left(afqmc_ctx* ctx, Walker* w, cudaStream_t st, int j, int s, int ell, double* U, double* tmp);

// Propagate the group's factors in Ucur ([walker][spin][N x nsm]) over nsl slices
// l = l_first, l_first + l_step, ... (right factors N x ns: B_l U; left factors ns x N: U B_l)
// with the fused kernel; lattices too large for it take the per-slice separable products.
static cudaError_t propagate(afqmc_ctx* ctx, Walker* w, cudaStream_t st, int left, int l_first, int l_step, int nsl) {
    const int N = w->N;
    PropArgs a;
    a.U0 = w->Ucur;
    a.sstride = w->fsz();
    a.wstride = 2 * w->fsz();
    for (int s = 0; s < 2; ++s) {
        a.nvec[s] = w->ns[s];
        a.vs[s] = left ? N : 1;
        a.es[s] = left ? 1 : w->ns[s];
        a.dplus[s] = exp(ctx->c[s]);
        a.dminus[s] = exp(-ctx->c[s]);
    }
    a.Ex = w->lat->Ex64;
    a.x = w->x;
    a.xstride = (long)ctx->p.M * N;
    a.L = w->L;
    a.l_first = l_first;
    a.l_step = l_step;
    a.nsl = nsl;
    a.left = left;
    a.nmat = 2 * w->nwk;
    cudaError_t e = launch_prop(st, a);
    if (e != cudaErrorInvalidValue) return e;
    cudaGetLastError();
    for (int t = 0; t < nsl; ++t)
        for (int j = 0; j < w->nwk; ++j)
            for (int s = 0; s < 2; ++s) {
                const int ell = l_first + t * l_step;
                double* U = w->Ucur + ((size_t)j * 2 + s) * w->fsz();
                e = left ? prop_left(ctx, w, st, j, s, ell, U, w->Utmp) : prop_right(ctx, w, st, j, s, ell, U, w->Utmp);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

// Spin groups for the batched FP64 steps: both spins in one launch when they have the same
// particle number, else one at a time.
static int spin_groups(const Walker* w, int grp[2][2], int ng[2]) {
    if (w->ns[0] == w->ns[1]) {
        grp[0][0] = 0;
        grp[0][1] = 1;
        ng[0] = 2;
        return 1;
    }
    grp[0][0] = 0;
    ng[0] = 1;
    grp[1][0] = 1;
    ng[1] = 1;
    return 2;
}

// A factor set of the group: matrix (walker j, spin s0 + q) at base + j wstride + (s0 + q) sstride
// for q < ng; layouts here always have wstride = 2 sstride, so the batch stride is uniform.
struct Fac {
    double* base;
    long wstride, sstride;
    double* at(int s0) const { return base + (size_t)s0 * sstride; }
    long bstride(int ng) const { return ng == 2 ? sstride : wstride; }
};
static Fac fac_cur(Walker* w) { return {w->Ucur, 2 * w->fsz(), w->fsz()}; }
static Fac fac_R(Walker* w, int j) { return {w->stackR(j), w->st_w(), w->st_s()}; }
static Fac fac_L(Walker* w, int j) { return {w->stackL(j), w->st_w(), w->st_s()}; }

static LuArgs lu_args(Walker* w, const Fac& f, int s0, int ng, long lda, int m, int n) {
    LuArgs a;
    a.A0 = f.at(s0);
    a.wstride = f.wstride;
    a.sstride = f.sstride;
    a.ng = ng;
    a.perm0 = w->perm2;
    a.flag0 = w->flag2;
    a.pstride = w->rows_max();
    a.lda = lda;
    a.m = m;
    a.n = n;
    a.nmat = w->nwk * ng;
    a.err = w->err;
    return a;
}

// Re-orthonormalisation (Sec. II.C): every right factor U (N x ns, row-major) of the spin group
// becomes P L from its partially pivoted LU, a basis of the same column space with entries of
// magnitude <= 1 (only the column space enters G, Eq. GrFMatNew).  sign[j] (nullable) is
// multiplied by the sign of the discarded triangular factor of walker j.
static cudaError_t stab_rows(afqmc_ctx* ctx, Walker* w, cudaStream_t st, const Fac& f, int s0, int ng, double* sign) {
    const int ns = w->ns[s0];
    LuArgs a = lu_args(w, f, s0, ng, ns, w->N, ns);
    cudaError_t e;
    {
        PhaseScope ps(ctx, AFQMC_PHASE_ELIM, st);
        if ((e = launch_lu(st, a)) != cudaSuccess) return e;
    }
    if (sign && (e = launch_lu_sign(st, a, 0, sign, w->visited)) != cudaSuccess) return e;
    return launch_lu_unit_rows(st, a);
}

// The same for left factors (ns x N): through their transposes.
static cudaError_t stab_cols(afqmc_ctx* ctx, Walker* w, cudaStream_t st, const Fac& f, int s0, int ng, double* sign) {
    const int N = w->N, ns = w->ns[s0], nmat = w->nwk * ng;
    const long bs = f.bstride(ng);
    cudaError_t e;
    count_launch();
    transpose_kernel<<<dim3(256, nmat), 256, 0, st>>>(f.at(s0), ns, N, w->Ut2, bs, w->fsz());
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const Fac t{w->Ut2, ng * w->fsz(), w->fsz()};
    if ((e = stab_rows(ctx, w, st, t, 0, ng, sign)) != cudaSuccess) return e;
    count_launch();
    transpose_kernel<<<dim3(256, nmat), 256, 0, st>>>(w->Ut2, N, ns, f.at(s0), w->fsz(), bs);
    return cudaGetLastError();
}

// Z[b] = (U_L U_R)^{-1} U_L (ns x N) for every (walker, spin) of a spin group (Eq. GrFMatNew):
// O = U_L U_R (FP64), its pivoted LU, then the substitutions with U_L as right-hand side.
// sign[j] (nullable) is multiplied by sign(det O) of walker j's spins.
// O = U_L U_R (FP64) for every (walker, spin) of a spin group, and its pivoted LU in place (Ob,
// perm2).  sign[j] (nullable) is multiplied by sign(det O) of walker j's spins.
static cudaError_t form_O(afqmc_ctx* ctx, Walker* w, cudaStream_t st, const Fac& R, const Fac& Lf, int s0, int ng,
                          double* sign) {
    const int N = w->N, ns = w->ns[s0], nmat = w->nwk * ng;
    const long os = (long)w->nsm * w->nsm;
    cudaError_t e;
    if (w->oz_Z) {
        OzGemmArgs o;
        o.M = ns; o.N = ns; o.K = N; o.batch = nmat;
        o.A = Lf.at(s0); o.lda = N; o.sA = Lf.bstride(ng);
        o.B = R.at(s0); o.ldb = ns; o.sB = R.bstride(ng);
        o.C = w->Ob; o.ldc = ns; o.sC = os;
        o.err = w->err;
        PhaseScope pd(ctx, AFQMC_PHASE_DGEMM, st);
        if ((e = ozaki_gemm(st, o, w->ozw, w->ozs)) != cudaSuccess) return e;
    } else {
        GemmArgs<double> g;
        g.M = ns; g.N = ns; g.K = N; g.batch = nmat;
        g.A = Lf.at(s0); g.lda = N; g.sA = Lf.bstride(ng);
        g.B = R.at(s0); g.ldb = ns; g.sB = R.bstride(ng);
        g.C = w->Ob; g.ldc = ns; g.sC = os;
        if ((e = gemm<double>(st, g)) != cudaSuccess) return e;
    }
    const Fac O{w->Ob, ng * os, os};
    LuArgs a = lu_args(w, O, 0, ng, ns, ns, ns);
    {
        PhaseScope ps(ctx, AFQMC_PHASE_LU_O, st);
        if ((e = launch_lu(st, a)) != cudaSuccess) return e;
    }
    if (sign && (e = launch_lu_sign(st, a, 1, sign, w->visited)) != cudaSuccess) return e;
    return cudaSuccess;
}

static cudaError_t form_Z(afqmc_ctx* ctx, Walker* w, cudaStream_t st, const Fac& R, const Fac& Lf, int s0, int ng,
                          double* sign) {
    const int N = w->N, ns = w->ns[s0], nmat = w->nwk * ng;
    const long os = (long)w->nsm * w->nsm, zs = (long)w->nsm * N;
    cudaError_t e;
    if ((e = form_O(ctx, w, st, R, Lf, s0, ng, sign)) != cudaSuccess) return e;
    if (w->Oinv) {
        // FP32 bulk: O^{-1} from the same LU (the solve with the identity in pivot order, ns
        // right-hand sides: the forward substitution of column c starts at row c), then
        // Z = O^{-1} U_L as an FP64-accurate digit-split product.  The forward error of Z is that of
        // the solve up to a factor of order one; the FP32 bulk keeps about seven digits of G.
        SolveArgs si;
        si.LU0 = w->Ob;
        si.ostride = os;
        si.perm0 = w->perm2;
        si.pstride = w->rows_max();
        si.eye = 1;  // the identity in pivot order, generated in the kernel
        si.ng = ng;
        si.Z0 = w->Oinv;
        si.zstride = os;
        si.ldl = ns;
        si.ns = ns;
        si.N = ns;
        si.nmat = nmat;
        {
            PhaseScope pv(ctx, AFQMC_PHASE_SOLVE, st);
            if ((e = launch_lu_solve(st, si)) != cudaSuccess) return e;
        }
        OzGemmArgs o;
        o.M = ns; o.N = N; o.K = ns; o.batch = nmat;
        o.A = w->Oinv; o.lda = ns; o.sA = os;
        o.B = Lf.at(s0); o.ldb = N; o.sB = Lf.bstride(ng);
        o.C = w->Z; o.ldc = N; o.sC = zs;
        o.err = w->err;
        PhaseScope pd(ctx, AFQMC_PHASE_DGEMM, st);
        return ozaki_gemm(st, o, w->ozw, w->ozs);
    }
    SolveArgs sa;
    sa.LU0 = w->Ob;
    sa.ostride = os;
    sa.perm0 = w->perm2;
    sa.pstride = w->rows_max();
    sa.B0 = Lf.at(s0);
    sa.wstride = Lf.wstride;
    sa.sstride = Lf.sstride;
    sa.ng = ng;
    sa.Z0 = w->Z;
    sa.zstride = zs;
    sa.ldl = ns;
    sa.ns = ns;
    sa.N = N;
    sa.nmat = nmat;
    PhaseScope pv(ctx, AFQMC_PHASE_SOLVE, st);
    return launch_lu_solve(st, sa);
}

// Gnew[b] (FP64, N x ld) = 1 - U_R Z[b] for the spin group of form_Z; then the drift against the
// bulk G (acc2 per walker, nullable) and the store into the bulk G.  The N x N product keeps
// FP64 accuracy for both bulk precisions (FP64 SIMT, or the digit-split tensor-core product):
// the LU bases are not orthonormal, so 1 - U_R Z cancels large terms and an FP32 product would
// lose the digits the recompute restores.
template <typename T>
static cudaError_t finish_G(afqmc_ctx* ctx, Walker* w, cudaStream_t st, const Fac& R, int s0, int ng, bool drift) {
    const int N = w->N, ns = w->ns[s0], nmat = w->nwk * ng;
    const long gs = (long)N * w->ld;
    cudaError_t e;
    if (w->oz_G) {
        OzGemmArgs o;
        o.M = N; o.N = N; o.K = ns; o.batch = nmat;
        o.A = R.at(s0); o.lda = ns; o.sA = R.bstride(ng);
        o.B = w->Z; o.ldb = N; o.sB = (long)w->nsm * N;
        o.C = w->Gnew; o.ldc = w->ld; o.sC = gs;
        o.err = w->err;
        PhaseScope pd(ctx, AFQMC_PHASE_DGEMM, st);
        if ((e = ozaki_gemm(st, o, w->ozw, w->ozs)) != cudaSuccess) return e;
    } else {
        GemmArgs<double> h;
        h.M = N; h.N = N; h.K = ns; h.batch = nmat;
        h.A = R.at(s0); h.lda = ns; h.sA = R.bstride(ng);
        h.B = w->Z; h.ldb = N; h.sB = (long)w->nsm * N;
        h.C = w->Gnew; h.ldc = w->ld; h.sC = gs;
        if ((e = gemm<double>(st, h)) != cudaSuccess) return e;
    }
    if ((e = launch_identity_minus<double>(st, w->Gnew, w->ld, N, nmat, gs)) != cudaSuccess) return e;
    T* Gb = (T*)w->G + (size_t)s0 * gs;                 // bulk G of (walker 0, spin s0)
    const long bs = (ng == 2) ? gs : 2 * gs;            // batch stride in the bulk G
    if (drift && (e = launch_drift<T>(st, Gb, (const T*)w->Gnew, w->ld, N, w->acc2, nmat, bs, gs, ng)) != cudaSuccess)
        return e;
    return launch_cast<T>(st, w->Gnew, w->ld, Gb, w->ld, N, N, nmat, gs, bs);
}

// ---------------------------------------------------------------------------
// T form (Sec. II.C: the walker carries U_R, U_L and T = (U_L U_R)^{-1}; G = 1 - U_R T U_L)
// ---------------------------------------------------------------------------
// The bulk T-form state from the FP64 factors after form_Z (Z = (U_L U_R)^{-1} U_L, ns x N): U_R = R,
// U_L = Z and T = (Z R)^{-1} = 1.  Any bases of the two spaces give the same G = 1 - U_R T U_L; this
// choice keeps the FP32 state accurate.  With the LU bases of the re-orthonormalisation and
// T = (U_L U_R)^{-1}, the FP32 product U_R T U_L cancels terms some 10^2 - 10^3 times larger than G
// (at 40 x 40, U = 6: |U_R| ~ 230, |U_L| ~ 140, |T| ~ 600, cond(U_L U_R) ~ 6e4), where
// U_R (U_L U_R)^{-1} U_L with the left factor taken as Z keeps FP32 rounding near 2e-6 (a numpy
// check on the same factors: 1.9e-6 against 4.5e-5).  The T form requires n_up = n_dn, so both
// spins form one group (ng = 2).
template <typename T>
static cudaError_t tform_set(afqmc_ctx* ctx, Walker* w, cudaStream_t st, const Fac& R) {
    (void)ctx;
    const int N = w->N, ns = w->nsm, nmat = 2 * w->nwk;
    const long os = (long)ns * ns;
    cudaError_t e;
    if ((e = launch_cast<T>(st, w->Ieye, ns, (T*)w->TT, ns, ns, ns, nmat, 0, os)) != cudaSuccess) return e;
    if ((e = launch_cast<T>(st, R.at(0), ns, (T*)w->TUR, ns, N, ns, nmat, R.bstride(2), (long)N * ns)) != cudaSuccess)
        return e;
    return launch_cast<T>(st, w->Z, N, (T*)w->TUL, N, ns, N, nmat, (long)ns * N, (long)N * ns);
}

// The bulk G of every walker from its T-form state: G = 1 - (U_R T) U_L, with U_R T in Tbuf.
template <typename T>
static cudaError_t tform_form_G(Walker* w, cudaStream_t st) {
    const int N = w->N, ns = w->nsm, nmat = 2 * w->nwk;
    const long fs = (long)N * ns;
    GemmArgs<T> g;
    g.M = N; g.N = ns; g.K = ns; g.batch = nmat;
    g.A = (const T*)w->TUR; g.lda = ns; g.sA = fs;
    g.B = (const T*)w->TT; g.ldb = ns; g.sB = (long)ns * ns;
    g.C = (T*)w->Tbuf; g.ldc = ns; g.sC = (long)N * w->ld;
    cudaError_t e = gemm<T>(st, g);
    if (e != cudaSuccess) return e;
    GemmArgs<T> h;
    h.M = N; h.N = N; h.K = ns; h.batch = nmat;
    h.A = (const T*)w->Tbuf; h.lda = ns; h.sA = (long)N * w->ld;
    h.B = (const T*)w->TUL; h.ldb = N; h.sB = fs;
    h.C = (T*)w->G; h.ldc = w->ld; h.sC = (long)N * w->ld;
    if ((e = gemm<T>(st, h)) != cudaSuccess) return e;
    if ((e = launch_identity_minus<T>(st, (T*)w->G, w->ld, N, nmat, (long)N * w->ld)) != cudaSuccess) return e;
    w->gvalid = true;
    return cudaSuccess;
}

// U (N x ns) <- B_l U for walker j, spin s, B_l = diag(exp(c_s x_l)) E.  E = Ex (x) Ex on the
// square lattice, so E U is two small products: along x for every row block y, then along y.
static cudaError_t prop_right(afqmc_ctx* ctx, Walker* w, cudaStream_t st, int j, int s, int ell, double* U,
                              double* tmp) {
    const int N = w->N, ns = w->ns[s], L = w->L;
    const int8_t* xl = w->x + (size_t)j * ctx->p.M * N + (size_t)(ell - 1) * N;
    cudaError_t e = launch_field_scales_T<double>(st, xl, N, ctx->c, w->d64, w->d64 + 2 * N, N);
    if (e != cudaSuccess) return e;
    GemmArgs<double> gx;  // tmp[(x,y), c] = sum_x' Ex[x, x'] U[(x',y), c]
    gx.M = L; gx.N = ns; gx.K = L; gx.batch = L;
    gx.A = w->lat->Ex64; gx.lda = L; gx.sA = 0;
    gx.B = U; gx.ldb = ns; gx.sB = (long)L * ns;
    gx.C = tmp; gx.ldc = ns; gx.sC = (long)L * ns;
    if ((e = gemm<double>(st, gx)) != cudaSuccess) return e;
    GemmArgs<double> gy;  // U[(x,y), c] = sum_y' Ex[y, y'] tmp[(x,y'), c]
    gy.M = L; gy.N = L * ns; gy.K = L;
    gy.A = w->lat->Ex64; gy.lda = L;
    gy.B = tmp; gy.ldb = (long)L * ns;
    gy.C = U; gy.ldc = (long)L * ns;
    if ((e = gemm<double>(st, gy)) != cudaSuccess) return e;
    return launch_scale_rows(st, U, N, ns, w->d64 + (size_t)s * N);
}

// U (ns x N) <- U B_l = (U diag(exp(c_s x_l))) E for walker j, spin s, with the same products.
static cudaError_t prop_left(afqmc_ctx* ctx, Walker* w, cudaStream_t st, int j, int s, int ell, double* U, double* tmp) {
    const int N = w->N, ns = w->ns[s], L = w->L;
    const int8_t* xl = w->x + (size_t)j * ctx->p.M * N + (size_t)(ell - 1) * N;
    cudaError_t e = launch_field_scales_T<double>(st, xl, N, ctx->c, w->d64, w->d64 + 2 * N, N);
    if (e != cudaSuccess) return e;
    if ((e = launch_scale_cols(st, U, ns, N, w->d64 + (size_t)s * N)) != cudaSuccess) return e;
    GemmArgs<double> gx;  // tmp[(a,y), x] = sum_x' U[a, (x',y)] Ex[x', x]
    gx.M = ns * L; gx.N = L; gx.K = L;
    gx.A = U; gx.lda = L;
    gx.B = w->lat->Ex64; gx.ldb = L;
    gx.C = tmp; gx.ldc = L;
    if ((e = gemm<double>(st, gx)) != cudaSuccess) return e;
    GemmArgs<double> gy;  // U[a, (x,y)] = sum_y' Ex[y, y'] tmp[(a,y'), x]
    gy.M = L; gy.N = L; gy.K = L; gy.batch = ns;
    gy.A = w->lat->Ex64; gy.lda = L; gy.sA = 0;
    gy.B = tmp; gy.ldb = L; gy.sB = N;
    gy.C = U; gy.ldc = L; gy.sC = N;
    return gemm<double>(st, gy);
}

// Copy the group's Ucur into stack entry j of URs (right) or ULs (left): one strided copy.
static cudaError_t to_stack(Walker* w, cudaStream_t st, bool right, int j) {
    double* dst = right ? w->stackR(j) : w->stackL(j);
    return cudaMemcpy2DAsync(dst, w->st_s() * 8, w->Ucur, w->fsz() * 8, w->fsz() * 8, 2 * (size_t)w->nwk,
                             cudaMemcpyDeviceToDevice, st);
}
static cudaError_t from_stack(Walker* w, cudaStream_t st, bool right, int j) {
    const double* src = right ? w->stackR(j) : w->stackL(j);
    return cudaMemcpy2DAsync(w->Ucur, w->fsz() * 8, src, w->st_s() * 8, w->fsz() * 8, 2 * (size_t)w->nwk,
                             cudaMemcpyDeviceToDevice, st);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
// FP32 bulk, G form: the most slices of propagation a stack basis carries between two
// re-orthonormalisations (the recompute may come more often; see afqmc_recompute_G).
constexpr int ORTHO_SLICES = 10;

extern "C" {

const char* afqmc_strerror(int code) {
    switch (code) {
        case AFQMC_OK: return "ok";
        case AFQMC_ERR_ARG: return "invalid argument";
        case AFQMC_ERR_OOM: return "device allocation failed";
        case AFQMC_ERR_CUDA: return "CUDA runtime error";
        case AFQMC_ERR_NUMERIC: return "non-finite ratio or singular matrix on the device";
        case AFQMC_ERR_TIMEOUT: return "a bounded device-side wait expired";
        case AFQMC_ERR_STATE: return "call out of sequence";
        case AFQMC_ERR_NODEV: return "no sm_103 device";
        default: return "unknown error";
    }
}

int afqmc_create(afqmc_ctx** out, const afqmc_params* p) {
    if (!out || !p) return AFQMC_ERR_ARG;
    *out = nullptr;
    if (p->M < 1 || p->stab_every < 1 || p->M % p->stab_every != 0) return AFQMC_ERR_ARG;
    if (p->precision != AFQMC_PREC_FP64 && p->precision != AFQMC_PREC_FP32) return AFQMC_ERR_ARG;
    if (!(p->dtau > 0.0)) return AFQMC_ERR_ARG;
    if (p->gemm < AFQMC_GEMM_TC3 || p->gemm > AFQMC_GEMM_TF32) return AFQMC_ERR_ARG;
    double lam;
    double c0, c1;
    if (p->hs == AFQMC_HS_SZ_REAL) {
        if (p->U < 0) return AFQMC_ERR_ARG;
        lam = acosh(exp(p->dtau * p->U / 2.0));
        c0 = lam; c1 = -lam;
    } else if (p->hs == AFQMC_HS_CHARGE_REAL) {
        if (p->U > 0) return AFQMC_ERR_ARG;
        lam = acosh(exp(p->dtau * fabs(p->U) / 2.0));
        c0 = lam; c1 = lam;
    } else {
        return AFQMC_ERR_ARG;
    }
    int dev = 0, major = 0, minor = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return AFQMC_ERR_NODEV;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (major != 10 || minor != 3) return AFQMC_ERR_NODEV;
    afqmc_ctx* ctx = new afqmc_ctx();
    ctx->p = *p;
    ctx->lam = lam;
    ctx->c[0] = c0;
    ctx->c[1] = c1;
    ctx->nsm = nsm;
    *out = ctx;
    return AFQMC_OK;
}

int afqmc_destroy(afqmc_ctx* ctx) {
    if (!ctx) return AFQMC_OK;
    cudaDeviceSynchronize();
    for (auto* w : ctx->w) {
        for (void* p : w->allocs) cudaFree(p);
        for (int q = 0; q < 2; ++q) {
            if (w->ev_chain[q]) cudaEventDestroy(w->ev_chain[q]);
            if (w->ev_prod[q]) cudaEventDestroy(w->ev_prod[q]);
        }
        if (w->ev_done) cudaEventDestroy(w->ev_done);
        if (w->ev_wrap) cudaEventDestroy(w->ev_wrap);
        if (w->ev_prop) cudaEventDestroy(w->ev_prop);
        if (w->ev_fork) cudaEventDestroy(w->ev_fork);
        if (w->ev_join) cudaEventDestroy(w->ev_join);
        if (w->ev_rc) cudaEventDestroy(w->ev_rc);
        for (auto& kv : w->graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (w->sf) cudaStreamDestroy(w->sf);
        if (w->sm) cudaStreamDestroy(w->sm);
        if (w->sp) cudaStreamDestroy(w->sp);
        delete w;
    }
    for (void* p : ctx->allocs) cudaFree(p);
    for (auto* l : ctx->lats) delete l;
    for (auto& pe : ctx->prof.pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    for (auto e : ctx->prof.pool) cudaEventDestroy(e);
    delete ctx;
    return AFQMC_OK;
}

int afqmc_init_walkers(afqmc_ctx* ctx, int n_walkers, const int* L, const int* n_up, const int* n_dn,
                       const double* P, const int8_t* fields, void* stream) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (n_walkers < 1 || !L || !n_up || !n_dn || !P || !ctx->w.empty()) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    const int M = ctx->p.M, S = ctx->p.stab_every, nst = M / S + 1;
    const size_t es = esize(ctx);
    for (int wi = 0; wi < n_walkers; ++wi) {
        if (L[wi] < 2 || L[wi] > 64) return AFQMC_ERR_ARG;
        int N = L[wi] * L[wi];
        if (n_up[wi] < 1 || n_up[wi] > N || n_dn[wi] < 1 || n_dn[wi] > N) return AFQMC_ERR_ARG;
        if (ctx->form == AFQMC_FORM_T && n_up[wi] != n_dn[wi]) return AFQMC_ERR_ARG;
    }
    // host offsets of every walker's trial state and fields in the caller's arrays
    std::vector<size_t> poff(n_walkers), foff(n_walkers);
    {
        size_t po = 0, fo = 0;
        for (int wi = 0; wi < n_walkers; ++wi) {
            const size_t N = (size_t)L[wi] * L[wi];
            poff[wi] = po;
            foff[wi] = fo;
            po += N * (n_up[wi] + n_dn[wi]);
            fo += (size_t)M * N;
        }
    }
    ctx->roff.assign(n_walkers, 0);
    for (int wi = 1; wi < n_walkers; ++wi) ctx->roff[wi] = ctx->roff[wi - 1] + 2 * (size_t)L[wi - 1] * L[wi - 1];
    // groups: walkers with the same (L, n_up, n_dn), in order of first appearance
    ctx->wmap.assign(n_walkers, {-1, -1});
    for (int wi = 0; wi < n_walkers; ++wi) {
        int g = -1;
        for (int q = 0; q < (int)ctx->w.size(); ++q) {
            Walker* w = ctx->w[q];
            if (w->L == L[wi] && w->ns[0] == n_up[wi] && w->ns[1] == n_dn[wi]) g = q;
        }
        if (g < 0) {
            Walker* w = new Walker();
            w->L = L[wi];
            w->ns[0] = n_up[wi];
            w->ns[1] = n_dn[wi];
            w->nwk = 0;
            ctx->w.push_back(w);
            g = (int)ctx->w.size() - 1;
        }
        Walker* w = ctx->w[g];
        ctx->wmap[wi] = {g, w->nwk};
        w->gid.push_back(wi);
        w->nwk++;
    }
    for (auto* w : ctx->w) {
        cudaError_t e;
        w->lat = get_lattice(ctx, w->L, st, &e);
        if (!w->lat) return fail(ctx, e);
        w->N = w->lat->N;
        w->ld = w->lat->ld;
        w->nsm = w->ns[0] > w->ns[1] ? w->ns[0] : w->ns[1];
        w->nst = nst;
        const int N = w->N, nsm = w->nsm, nwk = w->nwk;
        const long ld = w->ld;
        const int NW = (ctx->p.precision == AFQMC_PREC_FP64) ? window_max<double>() : window_max<float>();
        const size_t maxr = (size_t)w->rows_max();
        auto& A = w->allocs;
        CK(dalloc(A, &w->gid_d, (size_t)nwk * sizeof(int)));
        CK(cudaMemcpyAsync(w->gid_d, w->gid.data(), (size_t)nwk * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(dalloc(A, (char**)&w->G, (size_t)nwk * 2 * N * ld * es));
        CK(dalloc(A, (char**)&w->Tbuf, (size_t)nwk * 2 * N * ld * es));
        CK(dalloc(A, &w->x, (size_t)nwk * M * N));
        CK(dalloc(A, &w->u, (size_t)nwk * 2 * N * 8));
        CK(dalloc(A, (char**)&w->dvec, (size_t)nwk * 4 * N * es));
        CK(dalloc(A, &w->d64, 4 * (size_t)N * 8));
        CK(dalloc(A, &w->dec, (size_t)nwk * 2 * N));
        CK(dalloc(A, &w->ratio, (size_t)nwk * 2 * N * 8));
        CK(dalloc(A, &w->stats, (size_t)nwk * 8 * sizeof(int)));
        CK(dalloc(A, &w->maxr, (size_t)nwk * 8));
        CK(dalloc(A, &w->sign, (size_t)nwk * 8));
        CK(dalloc(A, &w->replay, (size_t)nwk * 2 * N));
        CK(dalloc(A, (char**)&w->colbuf, 4 * (size_t)N * es));  // [2 buffers][2 spins][N]
        CK(dalloc(A, (char**)&w->rowbuf, 4 * (size_t)N * es));
        CK(dalloc(A, &w->bar, sizeof(GridBar)));
        CK(dalloc(A, &w->err, sizeof(int)));
        for (int q = 0; q < 2; ++q) {
            CK(dalloc(A, &w->wm[q], (size_t)nwk * sizeof(int)));
            CK(dalloc(A, &w->widx[q], (size_t)nwk * NW * sizeof(int)));
            CK(dalloc(A, &w->wdtot[q], (size_t)nwk * 2 * NW * 8));
            CK(dalloc(A, (char**)&w->Wm[q], (size_t)nwk * 2 * NW * NW * es));
            CK(dalloc(A, (char**)&w->Wx[q], (size_t)nwk * 2 * NW * NW * es));
            CK(dalloc(A, (char**)&w->X[q], (size_t)nwk * 2 * N * NW * es));
            CK(dalloc(A, (char**)&w->Y[q], (size_t)nwk * 4 * NW * N * es));
            CK(dalloc(A, (char**)&w->snap[q], (size_t)nwk * 2 * NW * NW * es));
            CK(cudaEventCreateWithFlags(&w->ev_chain[q], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&w->ev_prod[q], cudaEventDisableTiming));
        }
        CK(cudaEventCreateWithFlags(&w->ev_done, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&w->ev_wrap, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&w->ev_prop, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&w->ev_join, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&w->ev_rc, cudaEventDisableTiming));
        {
            int lo = 0, hi = 0;
            CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            CK(cudaStreamCreateWithPriority(&w->sf, cudaStreamNonBlocking, lo));
            // the group's main stream (the accept chain, the wrap, the recompute) outranks the flush
            // and propagation streams, so their blocks never hold back a window kernel's launch
            CK(cudaStreamCreateWithPriority(&w->sm, cudaStreamNonBlocking, hi));
            CK(cudaStreamCreateWithPriority(&w->sp, cudaStreamNonBlocking, lo));
        }
        CK(dalloc(A, &w->visit_d, sizeof(unsigned long long)));
        CK(cudaMemsetAsync(w->visit_d, 0, sizeof(unsigned long long), st));
        CK(dalloc(A, &w->URs, (size_t)nwk * 2 * nst * N * nsm * 8));
        CK(dalloc(A, &w->ULs, (size_t)nwk * 2 * nst * N * nsm * 8));
        CK(dalloc(A, &w->Ucur, (size_t)nwk * 2 * N * nsm * 8));
        CK(dalloc(A, &w->Utmp, (size_t)N * nsm * 8));
        CK(dalloc(A, &w->Ut2, (size_t)nwk * 2 * N * nsm * 8));
        CK(dalloc(A, &w->Ob, (size_t)nwk * 2 * nsm * nsm * 8));
        CK(dalloc(A, &w->Z, (size_t)nwk * 2 * nsm * N * 8));
        CK(dalloc(A, &w->Gnew, (size_t)nwk * 2 * N * ld * 8));
        CK(dalloc(A, (char**)&w->perm2, (size_t)nwk * 2 * maxr * sizeof(int)));
        CK(dalloc(A, (char**)&w->flag2, (size_t)nwk * 2 * maxr));
        CK(dalloc(A, (char**)&w->visited, (size_t)nwk * maxr * sizeof(int)));
        CK(dalloc(A, &w->acc2, (size_t)nwk * 2 * 8));
        if (ctx->form == AFQMC_FORM_T) {
            const size_t fsb = (size_t)nwk * 2 * N * nsm * es, pan = (size_t)nwk * 2 * NW * nsm * es;
            CK(dalloc(A, (char**)&w->TUR, fsb));
            CK(dalloc(A, (char**)&w->TUL, fsb));
            CK(dalloc(A, (char**)&w->TT, (size_t)nwk * 2 * nsm * nsm * es));
            void** pans[] = {&w->ULI, &w->URI, &w->Vt, &w->Yt, &w->Ypt, &w->Pt};
            for (void** p : pans) {
                CK(dalloc(A, (char**)p, pan));
                CK(cudaMemsetAsync(*p, 0, pan, st));
            }
            std::vector<double> eye((size_t)nsm * nsm, 0.0);
            for (int i = 0; i < nsm; ++i) eye[(size_t)i * nsm + i] = 1.0;
            CK(dalloc(A, &w->Ieye, eye.size() * 8));
            CK(cudaMemcpyAsync(w->Ieye, eye.data(), eye.size() * 8, cudaMemcpyHostToDevice, st));
            CK(cudaStreamSynchronize(st));  // the host identity goes out of scope
        }
        if (ctx->p.gemm != AFQMC_GEMM_SIMT) {
            w->oz_Z = ozaki_pays(nsm, nsm, N, 2 * nwk);
            w->oz_G = ozaki_pays(N, N, nsm, 2 * nwk);
            const bool inv = ctx->form != AFQMC_FORM_T && ctx->p.precision == AFQMC_PREC_FP32 && w->oz_Z &&
                             w->oz_G && ozaki_pays(nsm, N, nsm, 2 * nwk);
            if (w->oz_Z || w->oz_G) {
                size_t f = ozaki_ws_bytes(nsm, nsm, N, 2 * nwk);
                f = std::max(f, ozaki_ws_bytes(N, N, nsm, 2 * nwk));
                if (inv) f = std::max(f, ozaki_ws_bytes(nsm, N, nsm, 2 * nwk));
                CK(dalloc(A, (char**)&w->ozw, f));
                CK(dalloc(A, &w->ozs, ozaki_sc_doubles(N > nsm ? N : nsm, N > nsm ? N : nsm, 2 * nwk) * 8));
            }
            if (inv) CK(dalloc(A, &w->Oinv, (size_t)nwk * 2 * nsm * nsm * 8));
        }
        CK(cudaMemsetAsync(w->err, 0, sizeof(int), st));
        CK(cudaMemsetAsync(w->dec, 0, (size_t)nwk * 2 * N, st));  // the block half stays 0 outside block FB
        CK(cudaMemsetAsync(w->ratio, 0, (size_t)nwk * 2 * N * 8, st));
        CK(cudaMemsetAsync(w->G, 0, (size_t)nwk * 2 * N * ld * es, st));
        CK(cudaMemsetAsync(w->Tbuf, 0, (size_t)nwk * 2 * N * ld * es, st));
        CK(cudaMemsetAsync(w->Gnew, 0, (size_t)nwk * 2 * N * ld * 8, st));
        for (int q = 0; q < 2; ++q) {
            CK(cudaMemsetAsync(w->Wm[q], 0, (size_t)nwk * 2 * NW * NW * es, st));
            CK(cudaMemsetAsync(w->Wx[q], 0, (size_t)nwk * 2 * NW * NW * es, st));
            CK(cudaMemsetAsync(w->X[q], 0, (size_t)nwk * 2 * N * NW * es, st));
            CK(cudaMemsetAsync(w->Y[q], 0, (size_t)nwk * 4 * NW * N * es, st));
        }
        // fields: the caller's, else Philox-drawn +-1 per walker
        for (int j = 0; j < nwk; ++j) {
            const int wi = w->gid[j];
            int8_t* xw = w->x + (size_t)j * M * N;
            if (fields) {
                CK(cudaMemcpyAsync(xw, fields + foff[wi], (size_t)M * N, cudaMemcpyHostToDevice, st));
            } else {
                count_launch();
                fields_kernel<<<(int)(((long)M * N + 255) / 256), 256, 0, st>>>(ctx->p.seed, (uint64_t)wi, (long)M * N, xw);
                CK(cudaGetLastError());
            }
        }
        count_launch();
        set_double_kernel<<<(nwk + 255) / 256, 256, 0, st>>>(w->sign, 1.0, nwk);
        CK(cudaGetLastError());
        // trial determinants -> stacks, G(0)  (Sec. II.B): P into URs entry 0 (N x ns), its
        // transpose starts the left stack, U_L(M) = P^T
        for (int j = 0; j < nwk; ++j)
            for (int s = 0; s < 2; ++s) {
                const double* Ph = P + poff[w->gid[j]] + (s ? (size_t)N * w->ns[0] : 0);
                CK(cudaMemcpyAsync(w->URs + ((size_t)j * 2 + s) * w->st_s(), Ph, (size_t)N * w->ns[s] * 8,
                                   cudaMemcpyHostToDevice, st));
            }
        for (int s = 0; s < 2; ++s) {
            count_launch();
            transpose_kernel<<<dim3(256, nwk), 256, 0, st>>>(w->URs + (size_t)s * w->st_s(), N, w->ns[s],
                                                            w->Ucur + (size_t)s * w->fsz(), w->st_w(), 2 * w->fsz());
            CK(cudaGetLastError());
        }
        int grp[2][2], ng[2];
        const int ngr = spin_groups(w, grp, ng);
        for (int gi = 0; gi < ngr; ++gi) {
            CK(stab_rows(ctx, w, st, fac_R(w, 0), grp[gi][0], ng[gi], w->sign));
            CK(stab_cols(ctx, w, st, fac_cur(w), grp[gi][0], ng[gi], w->sign));
        }
        CK(to_stack(w, st, false, M / S));
        // U_L(l - 1) = U_L(l) B_l, re-orthonormalised and stored at every recompute point
        for (int jj = M / S; jj >= 1; --jj) {
            CK(propagate(ctx, w, st, 1, jj * S, -1, S));  // slices jj S .. (jj - 1) S + 1
            for (int gi = 0; gi < ngr; ++gi) CK(stab_cols(ctx, w, st, fac_cur(w), grp[gi][0], ng[gi], w->sign));
            CK(to_stack(w, st, false, jj - 1));
        }
        // G(0) = 1 - U_R (U_L U_R)^{-1} U_L
        for (int gi = 0; gi < ngr; ++gi) {
            CK(form_Z(ctx, w, st, fac_R(w, 0), fac_L(w, 0), grp[gi][0], ng[gi], w->sign));
            if (ctx->p.precision == AFQMC_PREC_FP64) CK(finish_G<double>(ctx, w, st, fac_R(w, 0), grp[gi][0], ng[gi], false));
            else CK(finish_G<float>(ctx, w, st, fac_R(w, 0), grp[gi][0], ng[gi], false));
        }
        // T form: U_R(0), U_L(0) = Z and T(0) = 1 (Z = (U_L U_R)^{-1} U_L is still in w->Z)
        if (ctx->form == AFQMC_FORM_T) {
            if (ctx->p.precision == AFQMC_PREC_FP64) CK(tform_set<double>(ctx, w, st, fac_R(w, 0)));
            else CK(tform_set<float>(ctx, w, st, fac_R(w, 0)));
        }
        w->gvalid = true;
        w->pos = 0;
        w->last_dir = -1;
        w->need_recompute = false;
        w->visit = 0;
    }
    CK(cudaStreamSynchronize(st));
    for (auto* w : ctx->w) {
        int r = read_dev_err(ctx, w);
        if (r) return r;
    }
    return AFQMC_OK;
}

}  // extern "C"

static size_t ctx_replay_offset(const afqmc_ctx* ctx, int walker) { return ctx->roff[walker]; }

// Record an event that work outside this stream (and outside a graph captured from it) waits on:
// during stream capture as an external event node, else a plain record.
static cudaError_t record_outside(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, st);
}

// One slice of the recompute's propagation, on stream sq after event ev (nullable): forward,
// the right factor R(slice) = B_slice R(slice - 1); backward, the left factor L(slice - 1) =
// L(slice) B_slice.  The first slice of an interval starts from its stack entry; a later slice
// continues only the chain it follows (else the recompute propagates the interval itself).
static cudaError_t prop_step(afqmc_ctx* ctx, Walker* w, int slice, int dir, cudaStream_t sq, cudaEvent_t ev) {
    const int S = ctx->p.stab_every;
    const bool first = dir > 0 ? ((slice - 1) % S == 0) : (slice % S == 0);
    const int prev = dir > 0 ? slice - 1 : slice;
    if (!first && !(w->prop_dir == dir && w->prop_pos == prev)) return cudaSuccess;
    cudaError_t e;
    if (ev && (e = cudaStreamWaitEvent(sq, ev, 0)) != cudaSuccess) return e;
    if (first && (e = from_stack(w, sq, dir > 0, dir > 0 ? (slice - 1) / S : slice / S)) != cudaSuccess) return e;
    if ((e = propagate(ctx, w, sq, dir > 0 ? 0 : 1, slice, 1, 1)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(w->ev_prop, sq)) != cudaSuccess) return e;
    w->prop_pos = dir > 0 ? slice : slice - 1;
    w->prop_dir = dir;
    return cudaSuccess;
}

template <typename T>
static int sweep_impl(afqmc_ctx* ctx, int gi, int ell, int dir, int mode, int k, int nb, const uint8_t* replay,
                      cudaStream_t st) {
    Walker* w = ctx->w[gi];
    const int N = w->N, nwk = w->nwk;
    const long ld = w->ld;
    T* G0 = (T*)w->G;
    T* G1 = G0 + (size_t)N * ld;
    T* Tb = (T*)w->Tbuf;
    int8_t* xl = w->x + (size_t)(ell - 1) * N;
    T* d = (T*)w->dvec;
    T* dinv = d + (size_t)nwk * 2 * N;
    const T* E = (const T*)w->lat->Eb;
    const T* Einv = (const T*)w->lat->Einvb;
    const int NW = window_max<T>();
    const uint8_t* rep = nullptr;
    Batch bt;
    bt.nwk = nwk;
    bt.gstride = w->gstride();
    bt.xstride = (long)ctx->p.M * N;
    const int nb2 = 2 * nwk;  // (walker, spin) batch of the G products
    {
        PhaseScope ps(ctx, AFQMC_PHASE_PREP, st);
        CK(launch_uniforms(st, ctx->p.seed, w->gid_d, w->visit_d, 2 * N, w->u, nwk));
        CK(cudaMemsetAsync(w->stats, 0, (size_t)nwk * 8 * sizeof(int), st));
        CK(cudaMemsetAsync(w->maxr, 0, (size_t)nwk * 8, st));
        if (replay) {
            std::vector<uint8_t> h((size_t)nwk * 2 * N);
            for (int j = 0; j < nwk; ++j)
                memcpy(h.data() + (size_t)j * 2 * N, replay + (size_t)ctx_replay_offset(ctx, w->gid[j]), 2 * (size_t)N);
            CK(cudaMemcpyAsync(w->replay, h.data(), h.size(), cudaMemcpyHostToDevice, st));
            CK(cudaStreamSynchronize(st));  // the host staging buffer goes out of scope
            rep = w->replay;
        }
    }
    const bool use_tc = (sizeof(T) == 4) && ctx->p.gemm != AFQMC_GEMM_SIMT;
    const int split3 = ctx->p.gemm != AFQMC_GEMM_TF32;
    auto wrap = [&](int direction) -> cudaError_t {
        PhaseScope ps(ctx, AFQMC_PHASE_WRAP, st);
        cudaError_t e = launch_field_scales_T<T>(st, xl, N, ctx->c, d, dinv, N, nwk, bt.xstride);
        if (e != cudaSuccess) return e;
        const bool sep = ctx->wrap_mode == AFQMC_WRAP_SEPARABLE ||
                         (ctx->wrap_mode < 0 && sep_available<T>(w->L, N));
        if (sep) {
            // E = Ex (x) Ex: two passes per product, in place, both spins of every walker
            SepArgs a1, a2;
            sep_wrap_passes(direction, G0, ld, (long)N * ld, w->L, nb2, w->lat->Ex64, w->lat->Exi64, d, dinv, N, &a1,
                            &a2);
            a1.w = a2.w = ctx->sep_tile;
            PhaseScope pg(ctx, AFQMC_PHASE_WRAP_GEMM, st);
            if ((e = launch_sep<T>(st, a1)) != cudaSuccess) return e;
            return launch_sep<T>(st, a2);
        }
        if (use_tc) {
            // E and Einv are symmetric, so both products are A * Bt^T with K-major operands:
            //   forward : S^T = (G Einv)^T ;  G = D (E S) D^{-1}
            //   backward: G <- D^{-1} G D ;  S^T = (G E)^T ;  G = Einv S
            const float* Ef = (const float*)E;
            const float* Eif = (const float*)Einv;
            float* Gf = (float*)G0;
            float* Tf = (float*)Tb;
            if (direction < 0) {
                e = launch_scale2<T>(st, G0, ld, N, (long)N * ld, dinv, d, nb2);
                if (e != cudaSuccess) return e;
            }
            TcGemmArgs t1;
            t1.M = N; t1.N = N; t1.K = N; t1.batch = nb2;
            t1.A = Gf; t1.lda = ld; t1.sA = (long)N * ld;
            t1.Bt = direction > 0 ? Eif : Ef; t1.ldb = ld; t1.sB = 0;
            t1.C = Tf; t1.ldc = ld; t1.sC = (long)N * ld; t1.c_trans = 1;
            t1.split3 = split3;
            t1.err = w->err;
            {
                PhaseScope pg(ctx, AFQMC_PHASE_WRAP_GEMM, st);
                if ((e = tc_gemm(st, t1)) != cudaSuccess) return e;
            }
            TcGemmArgs t2;
            t2.M = N; t2.N = N; t2.K = N; t2.batch = nb2;
            t2.A = direction > 0 ? Ef : Eif; t2.lda = ld; t2.sA = 0;
            t2.Bt = Tf; t2.ldb = ld; t2.sB = (long)N * ld;
            t2.C = Gf; t2.ldc = ld; t2.sC = (long)N * ld;
            if (direction > 0) {
                t2.rs = (const float*)d; t2.srs = N;
                t2.cs = (const float*)dinv; t2.scs = N;
            }
            t2.split3 = split3;
            t2.err = w->err;
            PhaseScope pg(ctx, AFQMC_PHASE_WRAP_GEMM, st);
            return tc_gemm(st, t2);
        }
        GemmArgs<T> g1, g2;
        g1.M = N; g1.N = N; g1.K = N; g1.batch = nb2;
        g1.ldb = ld; g1.sB = (long)N * ld;
        g1.C = Tb; g1.ldc = ld; g1.sC = (long)N * ld;
        g1.lda = ld; g1.sA = 0;
        g2 = g1;
        if (direction > 0) {
            // Tb = E G ; G = D (Tb Einv) D^{-1}
            g1.A = E; g1.B = G0;
            g2.A = Tb; g2.sA = (long)N * ld;
            g2.B = Einv; g2.sB = 0;
            g2.C = G0;
            g2.rs = d; g2.srs = N;
            g2.cs = dinv; g2.scs = N;
        } else {
            // Tb = Einv D^{-1} G D ; G = Tb E
            g1.A = Einv; g1.B = G0;
            g1.bs = dinv; g1.sbs = N;
            g1.cs = d; g1.scs = N;
            g2.A = Tb; g2.sA = (long)N * ld;
            g2.B = E; g2.sB = 0;
            g2.C = G0;
        }
        {
            PhaseScope pg(ctx, AFQMC_PHASE_WRAP_GEMM, st);
            e = gemm<T>(st, g1);
        }
        if (e != cudaSuccess) return e;
        PhaseScope pg(ctx, AFQMC_PHASE_WRAP_GEMM, st);
        return gemm<T>(st, g2);
    };
    if (dir > 0) {
        CK(wrap(+1));
        CK(record_outside(w->ev_wrap, st));
    }
    SiteParams sp;
    sp.N = N;
    sp.ld = ld;
    sp.c[0] = ctx->c[0];
    sp.c[1] = ctx->c[1];
    sp.lam = ctx->lam;
    sp.hs = ctx->p.hs;
    sp.seed = ctx->p.seed;
    sp.walker = (uint64_t)w->gid[0];
    sp.visit = w->visit;
    for (int s = 0; s < 2; ++s)
        for (int xi = 0; xi < 2; ++xi) {
            const double x = xi == 0 ? 1.0 : -1.0;
            sp.dflip[s][xi] = exp(-2.0 * ctx->c[s] * x) - 1.0;
            sp.dstrip[s][xi] = exp(-ctx->c[s] * x) - 1.0;
        }
    for (int xi = 0; xi < 2; ++xi) {
        const double x = xi == 0 ? 1.0 : -1.0;
        sp.sflip[xi] = (ctx->p.hs == AFQMC_HS_CHARGE_REAL) ? exp(2.0 * ctx->lam * x) : 1.0;
    }
    SliceOut so;
    so.dec = w->dec;
    so.ratio = w->ratio;
    so.stats = w->stats;
    so.maxr = w->maxr;
    so.sign = w->sign;
    if (mode == AFQMC_MODE_LOCAL) {
        // one persistent cooperative launch per walker (its grid barriers are walker-wide)
        PhaseScope ps(ctx, AFQMC_PHASE_LOCAL, st);
        for (int j = 0; j < nwk; ++j) {
            SliceOut sj = so;
            sj.dec += (size_t)j * 2 * N;
            sj.ratio += (size_t)j * 2 * N;
            sj.stats += (size_t)j * 8;
            sj.maxr += j;
            sj.sign += j;
            SiteParams spj = sp;
            spj.walker = (uint64_t)w->gid[j];
            T* Gj = G0 + (size_t)j * bt.gstride;
            CK(cudaMemsetAsync(w->bar, 0, sizeof(GridBar), st));
            CK(launch_local<T>(st, Gj, Gj + (size_t)N * ld, xl + (size_t)j * bt.xstride, w->u + (size_t)j * 2 * N,
                               rep ? rep + (size_t)j * 2 * N : nullptr, spj, sj, (T*)w->colbuf, (T*)w->rowbuf, w->bar,
                               w->err, ctx->nsm));
        }
    } else {
        int nw = (mode == AFQMC_MODE_DELAYED) ? k : (NW / nb) * nb;
        // Window w's decisions and the corrected block of window w + 1 run on st; window w's
        // panels and rank-m product run on the group's flush stream sf and overlap the
        // decisions of window w + 1.  Before building window w + 1's block, st waits for the
        // product of window w - 1 (ev_prod), which is also what frees the window buffers of
        // parity (w + 1) & 1 for reuse.  Every launch covers all walkers of the group.
        WindowBufs wb[2];
        for (int q = 0; q < 2; ++q) {
            wb[q].m = w->wm[q];
            wb[q].idx = w->widx[q];
            wb[q].dtot = w->wdtot[q];
            wb[q].Wm = w->Wm[q];
            wb[q].Wx = w->Wx[q];
            wb[q].X = w->X[q];
            wb[q].Y = w->Y[q];
            wb[q].nwk = nwk;
        }
        PhaseScope ps(ctx, AFQMC_PHASE_CHAIN, st);
        int wi = 0;
        for (int s0 = 0; s0 < N; s0 += nw, ++wi) {
            const int n = (N - s0 < nw) ? N - s0 : nw;
            const int par = wi & 1;
            const T* blk = (wi > 0) ? (const T*)w->snap[par ^ 1] : nullptr;
            CK(launch_window_chain<T>(st, mode, G0, G1, xl, w->u, rep, sp, so, s0, n, nb, wb[par], blk, w->err, bt));
            const int sn = s0 + n, nn = (sn < N) ? ((N - sn < nw) ? N - sn : nw) : 0;
            if (nn > 0) {  // the next window's block
                if (wi > 0) CK(cudaStreamWaitEvent(st, w->ev_prod[par ^ 1], 0));
                CK(launch_next_block<T>(st, G0, G1, sp, wb[par], sn, nn, (T*)w->snap[par], bt));
            }
            CK(cudaEventRecord(w->ev_chain[par], st));
            CK(cudaStreamWaitEvent(w->sf, w->ev_chain[par], 0));
            PhaseScope pf(ctx, AFQMC_PHASE_FLUSH, w->sf);
            CK(launch_flush_panels<T>(w->sf, G0, G1, sp, wb[par], n, bt));
            {
                PhaseScope pg(ctx, AFQMC_PHASE_FLUSH_GEMM, w->sf);
                CK(launch_flush_gemm<T>(w->sf, G0, G1, sp, wb[par], n, bt));
            }
            CK(cudaEventRecord(w->ev_prod[par], w->sf));
        }
        CK(cudaEventRecord(w->ev_done, w->sf));
        CK(cudaStreamWaitEvent(st, w->ev_done, 0));
    }
    if (dir < 0) {
        CK(wrap(-1));
        CK(record_outside(w->ev_wrap, st));
    }
    CK(launch_bump(st, w->visit_d));
    return AFQMC_OK;
}

// One slice of the T form (Sec. II.C, Sec. III.A-B) for walker group gi, on stream st:
//   wrap   U_R <- D E U_R, U_L <- U_L E^{-1} D^{-1} (forward; backward the inverse moves after the
//          update) by the separable passes on the N x Nsigma and Nsigma x N factors; T is unchanged;
//   per window of sites J: the block 1 - U_R[J, :] T U_L[:, J] of G, the window kernel (the same
//          decisions, ratios and update matrix W as the G form), then the window's update
//          T <- T - V W Y with V = T U_L[:, I], Y = U_R[I, :] T (the G form's W by the push-through
//          identity, Eq. BlkFrcBsTnew2) and the rows I of U_R scaled by the field change
//          (Eq. UpdateLTRMat).
// ---- constrained-path AFQMC helpers (Sec. IV.D) ----
// la[z] = ln |det O_z| of the O = U_L U_R factored by launch_lu (U entries at the pivot rows).
__global__ void cp_logdet_kernel(const double* O0, long os, const int* perm0, long ps, int ns, double* la) {
    const int z = blockIdx.x;
    const double* O = O0 + (size_t)z * os;
    const int* perm = perm0 + (size_t)z * ps;
    double acc = 0.0;
    for (int c = threadIdx.x; c < ns; c += blockDim.x) acc += log(fabs(O[(size_t)perm[c] * ns + c]));
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        la[z] = s;
    }
}

// Start of a step: clear the per-step sums (the removed flag stays) and the sign accumulator.
__global__ void cp_begin_kernel(double* cpl, double* sg, int nwk) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nwk) return;
    cpl[4 * j + 0] = 0.0;
    cpl[4 * j + 1] = 0.0;
    cpl[4 * j + 3] = 0.0;
    sg[j] = 1.0;
}

// After the kinetic step's fresh determinant: the kinetic ln ratio against the tracked one, the
// constraint (the overlap keeps the sign sref it had when the walker's basis was last set), and the
// new tracked value.  set_ref (a new basis): only take the determinant and its sign as the reference.
__global__ void cp_kinetic_kernel(double* cpl, double* det, const double* la, const double* sg, double* sref,
                                  int nwk, int set_ref) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nwk) return;
    const double now = la[2 * j] + la[2 * j + 1];
    if (set_ref) {
        sref[j] = sg[j];
    } else {
        cpl[4 * j + 3] = now - det[j];
        if (!(sg[j] * sref[j] > 0.0)) cpl[4 * j + 2] = 1.0;
    }
    det[j] = now;
}

// End of a step: the tracked determinant follows the fields' ratios; out[j] = the step's ln weight
// factor (-inf for a removed walker).
__global__ void cp_finish_kernel(double* cpl, double* det, double* out, int nwk) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nwk) return;
    det[j] += cpl[4 * j + 1];
    out[j] = cpl[4 * j + 2] != 0.0 ? -INFINITY : cpl[4 * j + 3] + cpl[4 * j + 0];
}

// The window loop of the T form over the N sites of slice ell (Sec. II.C): per window J the block
// 1 - (U_R[J, :] T) U_L[:, J], the window kernel (Metropolis modes, or the constrained-path heat bath
// WIN_MODE_CP), then T <- T - (T U_L[:, I]) (W (U_R[I, :] T)) and the rows I of U_R times
// exp(mul c_s x'_I) (mul = 2 for a flip, 1 for a field set from none).
template <typename T>
static int tform_windows(afqmc_ctx* ctx, Walker* w, cudaStream_t st, int8_t* xl, int mode, int k, int nb,
                         const SiteParams& sp, const uint8_t* rep, double* cp, double mul) {
    const int N = w->N, nwk = w->nwk, ns = w->nsm, nb2 = 2 * nwk;
    const int NW = window_max<T>();
    const long fs = (long)N * ns;
    T* UR = (T*)w->TUR;
    T* UL = (T*)w->TUL;
    T* TT = (T*)w->TT;
    Batch bt;
    bt.nwk = nwk;
    bt.gstride = w->gstride();
    bt.xstride = (long)ctx->p.M * N;
    const double cm[2] = {mul * 0.5 * ctx->c[0], mul * 0.5 * ctx->c[1]};  // the scaling kernel applies exp(2 c x)
    SliceOut so;
    so.dec = w->dec;
    so.ratio = w->ratio;
    so.stats = w->stats;
    so.maxr = w->maxr;
    so.sign = w->sign;
    so.cp = cp;
    WindowBufs wb;
    wb.m = w->wm[0];
    wb.idx = w->widx[0];
    wb.dtot = w->wdtot[0];
    wb.Wm = w->Wm[0];
    wb.Wx = w->Wx[0];
    wb.X = w->X[0];
    wb.Y = w->Y[0];
    wb.nwk = nwk;
    T* blk = (T*)w->snap[0];          // [nwk][2][NW x NW]: the window's block of G
    T* P = (T*)w->Pt;                 // [nwk][2][NW x ns]: U_R[J, :] T
    T* ULI = (T*)w->ULI;              // [nwk][2][ns x NW]
    T* URI = (T*)w->URI;              // [nwk][2][NW x ns]
    T* V = (T*)w->Vt;                 // [nwk][2][ns x NW]
    T* Y = (T*)w->Yt;                 // [nwk][2][NW x ns]
    T* Yp = (T*)w->Ypt;               // [nwk][2][NW x ns]
    const long sB = (long)NW * NW, sP = (long)NW * ns, sT = (long)ns * ns;
    {
        PhaseScope ps(ctx, AFQMC_PHASE_CHAIN, st);
        const int nw = (mode == AFQMC_MODE_BLOCKFB || mode == WIN_MODE_CPB) ? (NW / nb) * nb : k;
        for (int s0 = 0; s0 < N; s0 += nw) {
            const int n = (N - s0 < nw) ? N - s0 : nw;
            // the window's block of G: 1 - (U_R[J, :] T) U_L[:, J]
            GemmArgs<T> g1;
            g1.M = n; g1.N = ns; g1.K = ns; g1.batch = nb2;
            g1.A = UR + (size_t)s0 * ns; g1.lda = ns; g1.sA = fs;
            g1.B = TT; g1.ldb = ns; g1.sB = sT;
            g1.C = P; g1.ldc = ns; g1.sC = sP;
            CK(gemm<T>(st, g1));
            GemmArgs<T> g2;
            g2.M = n; g2.N = n; g2.K = ns; g2.batch = nb2;
            g2.A = P; g2.lda = ns; g2.sA = sP;
            g2.B = UL + s0; g2.ldb = N; g2.sB = fs;
            g2.C = blk; g2.ldc = NW; g2.sC = sB;
            CK(gemm<T>(st, g2));
            CK(launch_identity_minus<T>(st, blk, NW, n, nb2, sB));
            // decisions and the window's W
            CK(launch_window_chain<T>(st, mode, (const T*)w->G, nullptr, xl, w->u, rep, sp, so, s0, n, nb, wb, blk,
                                      w->err, bt));
            // T <- T - (T U_L[:, I]) (W (U_R[I, :] T)), then the rows I of U_R
            PhaseScope pf(ctx, AFQMC_PHASE_FLUSH, st);
            CK(launch_tform_gather<T>(st, UR, UL, N, ns, ns, fs, fs, wb, ULI, URI, nb2));
            GemmArgs<T> v;
            v.M = ns; v.N = NW; v.K = ns; v.batch = nb2;
            v.A = TT; v.lda = ns; v.sA = sT;
            v.B = ULI; v.ldb = NW; v.sB = (long)ns * NW;
            v.C = V; v.ldc = NW; v.sC = (long)ns * NW;
            CK(gemm<T>(st, v));
            GemmArgs<T> y;
            y.M = NW; y.N = ns; y.K = ns; y.batch = nb2;
            y.A = URI; y.lda = ns; y.sA = sP;
            y.B = TT; y.ldb = ns; y.sB = sT;
            y.C = Y; y.ldc = ns; y.sC = sP;
            CK(gemm<T>(st, y));
            GemmArgs<T> yp;  // Y' = W Y over the m accepted rows
            yp.M = NW; yp.N = ns; yp.K = NW; yp.Kdev = wb.m; yp.kdiv = 2; yp.batch = nb2;
            yp.A = (const T*)wb.Wx; yp.lda = NW; yp.sA = sB;
            yp.B = Y; yp.ldb = ns; yp.sB = sP;
            yp.C = Yp; yp.ldc = ns; yp.sC = sP;
            CK(gemm<T>(st, yp));
            GemmArgs<T> t;  // T -= V Y'
            t.M = ns; t.N = ns; t.K = NW; t.Kdev = wb.m; t.kdiv = 2; t.batch = nb2;
            t.A = V; t.lda = NW; t.sA = (long)ns * NW;
            t.B = Yp; t.ldb = ns; t.sB = sP;
            t.C = TT; t.ldc = ns; t.sC = sT;
            t.alpha = T(-1); t.beta = T(1);
            {
                PhaseScope pg(ctx, AFQMC_PHASE_FLUSH_GEMM, st);
                CK(gemm<T>(st, t));
            }
            CK(launch_tform_scale_rows<T>(st, UR, N, ns, ns, fs, wb, xl, bt.xstride, cm, nb2));
        }
    }
    return AFQMC_OK;
}

template <typename T>
static int sweep_impl_T(afqmc_ctx* ctx, int gi, int ell, int dir, int mode, int k, int nb, const uint8_t* replay,
                        cudaStream_t st) {
    Walker* w = ctx->w[gi];
    const int N = w->N, nwk = w->nwk, ns = w->nsm, nb2 = 2 * nwk;
    int8_t* xl = w->x + (size_t)(ell - 1) * N;
    T* d = (T*)w->dvec;
    T* dinv = d + (size_t)nwk * 2 * N;
    const int NW = window_max<T>();
    const long fs = (long)N * ns;
    T* UR = (T*)w->TUR;
    T* UL = (T*)w->TUL;
    const uint8_t* rep = nullptr;
    Batch bt;
    bt.nwk = nwk;
    bt.gstride = w->gstride();
    bt.xstride = (long)ctx->p.M * N;
    w->gvalid = false;
    {
        PhaseScope ps(ctx, AFQMC_PHASE_PREP, st);
        CK(launch_uniforms(st, ctx->p.seed, w->gid_d, w->visit_d, 2 * N, w->u, nwk));
        CK(cudaMemsetAsync(w->stats, 0, (size_t)nwk * 8 * sizeof(int), st));
        CK(cudaMemsetAsync(w->maxr, 0, (size_t)nwk * 8, st));
        if (replay) {
            std::vector<uint8_t> h((size_t)nwk * 2 * N);
            for (int j = 0; j < nwk; ++j)
                memcpy(h.data() + (size_t)j * 2 * N, replay + (size_t)ctx_replay_offset(ctx, w->gid[j]), 2 * (size_t)N);
            CK(cudaMemcpyAsync(w->replay, h.data(), h.size(), cudaMemcpyHostToDevice, st));
            CK(cudaStreamSynchronize(st));
            rep = w->replay;
        }
    }
    auto wrap = [&](int direction) -> cudaError_t {
        PhaseScope ps(ctx, AFQMC_PHASE_WRAP, st);
        cudaError_t e = launch_field_scales_T<T>(st, xl, N, ctx->c, d, dinv, N, nwk, bt.xstride);
        if (e != cudaSuccess) return e;
        SepArgs r, l;
        r.L = l.L = w->L;
        r.N = l.N = N;
        r.batch = l.batch = nb2;
        r.C = l.C = ns;
        r.sv = l.sv = N;
        r.w = l.w = ctx->sep_tile;
        r.G = UR; r.ld = ns; r.sG = fs; r.side = 0;
        l.G = UL; l.ld = N; l.sG = fs; l.side = 1;
        if (direction > 0) {  // U_R <- D (E U_R), U_L <- (U_L E^{-1}) D^{-1}
            r.A = w->lat->Ex64; r.rs_out = d;
            l.A = w->lat->Exi64; l.cs_out = dinv;
        } else {              // U_R <- E^{-1} (D^{-1} U_R), U_L <- (U_L D) E
            r.A = w->lat->Exi64; r.rs_in = dinv;
            l.A = w->lat->Ex64; l.cs_in = d;
        }
        PhaseScope pg(ctx, AFQMC_PHASE_WRAP_GEMM, st);
        if ((e = launch_sep<T>(st, r)) != cudaSuccess) return e;
        return launch_sep<T>(st, l);
    };
    if (dir > 0) {
        CK(wrap(+1));
        CK(record_outside(w->ev_wrap, st));
    }
    SiteParams sp;
    sp.N = N;
    sp.ld = w->ld;
    sp.c[0] = ctx->c[0];
    sp.c[1] = ctx->c[1];
    sp.lam = ctx->lam;
    sp.hs = ctx->p.hs;
    sp.seed = ctx->p.seed;
    sp.walker = (uint64_t)w->gid[0];
    sp.visit = w->visit;
    for (int s = 0; s < 2; ++s)
        for (int xi = 0; xi < 2; ++xi) {
            const double x = xi == 0 ? 1.0 : -1.0;
            sp.dflip[s][xi] = exp(-2.0 * ctx->c[s] * x) - 1.0;
            sp.dstrip[s][xi] = exp(-ctx->c[s] * x) - 1.0;
        }
    for (int xi = 0; xi < 2; ++xi) {
        const double x = xi == 0 ? 1.0 : -1.0;
        sp.sflip[xi] = (ctx->p.hs == AFQMC_HS_CHARGE_REAL) ? exp(2.0 * ctx->lam * x) : 1.0;
    }
    {
        const int rc = tform_windows<T>(ctx, w, st, xl, mode, k, nb, sp, rep, nullptr, 2.0);
        if (rc) return rc;
    }
    if (dir < 0) {
        CK(wrap(-1));
        CK(record_outside(w->ev_wrap, st));
    }
    CK(launch_bump(st, w->visit_d));
    return AFQMC_OK;
}

extern "C" {

int afqmc_sweep_slice(afqmc_ctx* ctx, int slice, int dir, int mode, int k, int nb, const uint8_t* replay,
                      afqmc_slice_stats* stats, void* stream) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (ctx->w.empty() || slice < 1 || slice > ctx->p.M || (dir != 1 && dir != -1)) return AFQMC_ERR_ARG;
    const bool f64 = ctx->p.precision == AFQMC_PREC_FP64;
    const int NW = f64 ? window_max<double>() : window_max<float>();
    if (mode == AFQMC_MODE_DELAYED && (k < 1 || k > NW)) return AFQMC_ERR_ARG;
    if (mode == AFQMC_MODE_BLOCKFB && (nb < 1 || nb > 32)) return AFQMC_ERR_ARG;
    if (mode != AFQMC_MODE_LOCAL && mode != AFQMC_MODE_DELAYED && mode != AFQMC_MODE_BLOCKFB) return AFQMC_ERR_ARG;
    if (ctx->form == AFQMC_FORM_T && mode == AFQMC_MODE_LOCAL) return AFQMC_ERR_ARG;  // k = 1 delayed is local
    for (auto* w : ctx->w) {
        if (w->need_recompute) return AFQMC_ERR_STATE;
        if (dir > 0 && w->pos != slice - 1) return AFQMC_ERR_STATE;
        if (dir < 0 && w->pos != slice) return AFQMC_ERR_STATE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    // Every group runs on its own high-priority stream forked from (and joined back into) st, so
    // groups run concurrently.  With graphs on, a group's slice is captured once per (slice, dir,
    // mode, k, nb) and then replayed: every launch of the slice, the flush stream's included, in
    // one graph launch.
    const bool use_graph = ctx->graphs && !replay && !ctx->prof.on && ctx->form == AFQMC_FORM_G;
    for (int gi = 0; gi < (int)ctx->w.size(); ++gi) {
        Walker* w = ctx->w[gi];
        CK(cudaEventRecord(w->ev_fork, st));
        CK(cudaStreamWaitEvent(w->sm, w->ev_fork, 0));
        cudaStream_t sg = w->sm;
        if (use_graph) {
            const long long key = ((((long long)slice * 4 + (dir > 0 ? 1 : 0)) * 4 + mode) * 512 + k) * 64 + nb;
            auto it = w->graphs.find(key);
            if (it == w->graphs.end()) {
                Walker::Graph gr;
                cudaGraph_t graph = nullptr;
                const long long l0 = afqmc_launch_count();
                CK(cudaStreamBeginCapture(sg, cudaStreamCaptureModeRelaxed));
                rc = f64 ? sweep_impl<double>(ctx, gi, slice, dir, mode, k, nb, nullptr, sg)
                         : sweep_impl<float>(ctx, gi, slice, dir, mode, k, nb, nullptr, sg);
                cudaError_t ec = cudaStreamEndCapture(sg, &graph);
                if (rc) {
                    if (graph) cudaGraphDestroy(graph);
                    return rc;
                }
                CK(ec);
                gr.launches = afqmc_launch_count() - l0;
                cudaError_t ei = cudaGraphInstantiate(&gr.exec, graph, 0);
                cudaGraphDestroy(graph);
                CK(ei);
                it = w->graphs.emplace(key, gr).first;
            } else {
                count_launch((int)it->second.launches);
            }
            CK(cudaGraphLaunch(it->second.exec, sg));
        } else if (ctx->form == AFQMC_FORM_T) {
            rc = f64 ? sweep_impl_T<double>(ctx, gi, slice, dir, mode, k, nb, replay, sg)
                     : sweep_impl_T<float>(ctx, gi, slice, dir, mode, k, nb, replay, sg);
            if (rc) return rc;
        } else {
            rc = f64 ? sweep_impl<double>(ctx, gi, slice, dir, mode, k, nb, replay, sg)
                     : sweep_impl<float>(ctx, gi, slice, dir, mode, k, nb, replay, sg);
            if (rc) return rc;
        }
        // the factor of the next recompute follows the sweep one slice behind, on sp, while the
        // chain runs (not during a wrap): forward, slice l's right-factor step waits for slice
        // l + 1's wrap; backward, slice l's left-factor step waits for slice l's own wrap down
        if (dir > 0) {
            if (w->pend_slice > 0) CK(prop_step(ctx, w, w->pend_slice, +1, w->sp, w->ev_wrap));
            w->pend_slice = slice;
        } else {
            w->pend_slice = 0;
            CK(prop_step(ctx, w, slice, -1, w->sp, w->ev_wrap));
        }
        if (sg != st) {
            CK(cudaEventRecord(w->ev_join, sg));
            CK(cudaStreamWaitEvent(st, w->ev_join, 0));
        }
        w->pos = (dir > 0) ? slice : slice - 1;
        w->last_dir = dir;
        w->visit++;
        if (w->pos % ctx->p.stab_every == 0) w->need_recompute = true;
    }
    if (stats) {
        CK(cudaStreamSynchronize(st));
        for (auto* w : ctx->w) {
            int r = read_dev_err(ctx, w);
            if (r) return r;
            std::vector<int> h((size_t)w->nwk * 8);
            std::vector<double> mr(w->nwk), sg(w->nwk);
            CK(cudaMemcpy(h.data(), w->stats, h.size() * sizeof(int), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(mr.data(), w->maxr, (size_t)w->nwk * 8, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(sg.data(), w->sign, (size_t)w->nwk * 8, cudaMemcpyDeviceToHost));
            for (int j = 0; j < w->nwk; ++j) {
                afqmc_slice_stats& o = stats[w->gid[j]];
                o.proposals = h[j * 8 + 0];
                o.accepts = h[j * 8 + 1];
                o.flipped = h[j * 8 + 2];
                o.flushes = h[j * 8 + 3];
                o.max_abs_ratio = mr[j];
                o.sign = sg[j];
            }
        }
    }
    return AFQMC_OK;
}

int afqmc_recompute_G(afqmc_ctx* ctx, double* rel_drift, void* stream) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (ctx->w.empty()) return AFQMC_ERR_ARG;
    const int S = ctx->p.stab_every;
    for (auto* w : ctx->w)
        if (w->pos % S != 0) return AFQMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    const bool f64 = ctx->p.precision == AFQMC_PREC_FP64;
    cudaStream_t st0 = st;
    for (auto* w : ctx->w) {
        const int j = w->pos / S;
        // groups recompute concurrently, each on its high-priority main stream
        CK(cudaEventRecord(w->ev_fork, st0));
        CK(cudaStreamWaitEvent(w->sm, w->ev_fork, 0));
        st = w->sm;
        PhaseScope ps(ctx, AFQMC_PHASE_RECOMPUTE, st);
        CK(cudaMemsetAsync(w->acc2, 0, (size_t)w->nwk * 16, st));
        // the factors of the current position: one side from the stacks, the other propagated
        // over the last S slices from the previous stack entry and re-orthonormalised.  With an
        // FP32 bulk G (G form) the re-orthonormalisation leaves the critical path: G is formed
        // from the propagated factor itself (at most ORTHO_SLICES slices from an orthonormal
        // basis, so its column scales spread by at most cond(B)^ORTHO_SLICES and G keeps far more
        // than FP32 accuracy; Eq. GrFMatNew holds for any basis of the same space), and the LU
        // that makes the stack entry, when one is due, runs afterwards on the propagation stream,
        // where the next interval's propagation starts from it.
        const bool fwd = w->last_dir > 0;
        const bool prop = fwd ? (j > 0) : (w->pos != ctx->p.M);
        const bool defer = prop && !f64 && ctx->form == AFQMC_FORM_G;
        int grp[2][2], ng[2];
        const int ngr = spin_groups(w, grp, ng);
        if (prop) {
            CK(cudaStreamWaitEvent(st, w->ev_prop, 0));
            if (fwd && w->pend_slice == w->pos) {  // the interval's last slice: its step on st now
                CK(prop_step(ctx, w, w->pend_slice, +1, st, nullptr));
                w->pend_slice = 0;
            }
            if (w->prop_pos != w->pos || w->prop_dir != w->last_dir) {  // not followed slice by slice
                CK(from_stack(w, st, fwd, fwd ? j - 1 : j + 1));
                if (fwd) CK(propagate(ctx, w, st, 0, w->pos - S + 1, 1, S));
                else CK(propagate(ctx, w, st, 1, w->pos + S, -1, S));
            }
            if (!defer) {
                for (int gi = 0; gi < ngr; ++gi) {
                    if (fwd) CK(stab_rows(ctx, w, st, fac_cur(w), grp[gi][0], ng[gi], nullptr));
                    else CK(stab_cols(ctx, w, st, fac_cur(w), grp[gi][0], ng[gi], nullptr));
                }
                CK(to_stack(w, st, fwd, j));
            }
        }
        if (ctx->form == AFQMC_FORM_T) {
            // the bulk factors from the FP64 ones (U_R, Z = (U_L U_R)^{-1} U_L, T = 1); with a drift
            // requested, G is formed from the bulk state first and compared with the recomputed FP64 G
            if (rel_drift) {
                if (f64) CK(tform_form_G<double>(w, st));
                else CK(tform_form_G<float>(w, st));
            }
            CK(form_Z(ctx, w, st, fac_R(w, j), fac_L(w, j), 0, 2, nullptr));
            if (rel_drift) {
                if (f64) CK(finish_G<double>(ctx, w, st, fac_R(w, j), 0, 2, true));
                else CK(finish_G<float>(ctx, w, st, fac_R(w, j), 0, 2, true));
            }
            if (f64) CK(tform_set<double>(ctx, w, st, fac_R(w, j)));
            else CK(tform_set<float>(ctx, w, st, fac_R(w, j)));
            w->gvalid = rel_drift != nullptr;
        } else {
            const Fac R = (defer && fwd) ? fac_cur(w) : fac_R(w, j);
            const Fac Lf = (defer && !fwd) ? fac_cur(w) : fac_L(w, j);
            for (int gi = 0; gi < ngr; ++gi) {
                CK(form_Z(ctx, w, st, R, Lf, grp[gi][0], ng[gi], nullptr));
                if (f64) CK(finish_G<double>(ctx, w, st, R, grp[gi][0], ng[gi], true));
                else CK(finish_G<float>(ctx, w, st, R, grp[gi][0], ng[gi], true));
            }
            if (defer) {  // the stack entry, off the critical path
                // Re-orthonormalise only when the next interval would otherwise propagate the basis
                // over more than ORTHO_SLICES slices: its column scales then spread by at most
                // cond(B)^ORTHO_SLICES, as at a recompute period of that length, which G formed in
                // FP64 from that basis absorbs far below FP32 rounding.
                if (w->orth_dir != w->last_dir) {
                    w->orth_dir = w->last_dir;
                    w->orth_since = 0;
                }
                w->orth_since += S;
                const bool ortho = w->orth_since + S > ORTHO_SLICES;
                CK(cudaEventRecord(w->ev_rc, st));
                CK(cudaStreamWaitEvent(w->sp, w->ev_rc, 0));
                if (ortho) {
                    for (int gi = 0; gi < ngr; ++gi) {
                        if (fwd) CK(stab_rows(ctx, w, w->sp, fac_cur(w), grp[gi][0], ng[gi], nullptr));
                        else CK(stab_cols(ctx, w, w->sp, fac_cur(w), grp[gi][0], ng[gi], nullptr));
                    }
                    w->orth_since = 0;
                }
                CK(to_stack(w, w->sp, fwd, j));
                CK(cudaEventRecord(w->ev_prop, w->sp));
            }
        }
        w->need_recompute = false;
        CK(cudaEventRecord(w->ev_join, st));
        CK(cudaStreamWaitEvent(st0, w->ev_join, 0));
    }
    st = st0;
    if (rel_drift) {
        CK(cudaStreamSynchronize(st));
        for (auto* w : ctx->w) {
            int r = read_dev_err(ctx, w);
            if (r) return r;
            std::vector<double> h((size_t)w->nwk * 2);
            CK(cudaMemcpy(h.data(), w->acc2, h.size() * 8, cudaMemcpyDeviceToHost));
            for (int jw = 0; jw < w->nwk; ++jw)
                rel_drift[w->gid[jw]] = h[2 * jw + 1] > 0 ? sqrt(h[2 * jw] / h[2 * jw + 1]) : 0.0;
        }
    }
    return AFQMC_OK;
}

// ---------------------------------------------------------------------------
// constrained-path AFQMC (Sec. IV.D) on the T-form walkers: U_R = phi_k, U_L = psi_T^+ fixed,
// T = (U_L U_R)^{-1}; fields drawn by the window kernel's heat bath (WIN_MODE_CP)
// ---------------------------------------------------------------------------
}  // extern "C"

static int cp_check(afqmc_ctx* ctx, bool need_init) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (ctx->form != AFQMC_FORM_T || ctx->p.precision != AFQMC_PREC_FP64 || ctx->w.size() != 1) return AFQMC_ERR_STATE;
    if (need_init && !ctx->w[0]->cp) return AFQMC_ERR_STATE;
    return AFQMC_OK;
}

// O = U_L U_R (FP64), its pivoted LU, ln |det| per matrix and the sign per walker, T = O^{-1}, and
// (cp_kinetic_kernel) the determinant bookkeeping.  set_ref: a new basis (init, re-orthonormalisation).
static int cp_refresh(afqmc_ctx* ctx, Walker* w, cudaStream_t st, int set_ref) {
    const int N = w->N, ns = w->nsm, nwk = w->nwk, nb2 = 2 * nwk;
    const long fs = (long)N * ns, os = (long)ns * ns;
    GemmArgs<double> g;
    g.M = ns; g.N = ns; g.K = N; g.batch = nb2;
    g.A = (const double*)w->TUL; g.lda = N; g.sA = fs;
    g.B = (const double*)w->TUR; g.ldb = ns; g.sB = fs;
    g.C = w->Ob; g.ldc = ns; g.sC = os;
    CK(gemm<double>(st, g));
    const Fac O{w->Ob, 2 * os, os};
    LuArgs a = lu_args(w, O, 0, 2, ns, ns, ns);
    CK(launch_lu(st, a));
    count_launch();
    cp_begin_kernel<<<(nwk + 127) / 128, 128, 0, st>>>(w->cpl, w->cpsg, nwk);  // (re)sets the sign product
    CK(cudaGetLastError());
    CK(launch_lu_sign(st, a, 1, w->cpsg, w->visited));
    count_launch();
    cp_logdet_kernel<<<nb2, 256, 0, st>>>(w->Ob, os, w->perm2, w->rows_max(), ns, w->cpla);
    CK(cudaGetLastError());
    SolveArgs sa;
    sa.LU0 = w->Ob; sa.ostride = os;
    sa.perm0 = w->perm2; sa.pstride = w->rows_max();
    sa.B0 = w->Ieye; sa.wstride = 0; sa.sstride = 0; sa.ng = 2;
    sa.Z0 = (double*)w->TT; sa.zstride = os;
    sa.ldl = ns; sa.ldb = ns; sa.ns = ns; sa.N = ns; sa.nmat = nb2;
    CK(launch_lu_solve(st, sa));
    count_launch();
    cp_kinetic_kernel<<<(nwk + 127) / 128, 128, 0, st>>>(w->cpl, w->cpdet, w->cpla, w->cpsg, w->cpsref, nwk, set_ref);
    CK(cudaGetLastError());
    return AFQMC_OK;
}

extern "C" {

int afqmc_cp_init(afqmc_ctx* ctx, const double* P, const double* phi0, void* stream) {
    int rc = cp_check(ctx, false);
    if (rc) return rc;
    if (!P) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    Walker* w = ctx->w[0];
    const int N = w->N, ns = w->nsm, nwk = w->nwk;
    const size_t fs = (size_t)N * ns;
    if (!w->cpl) {
        std::vector<void*>& A = w->allocs;
        CK(dalloc(A, &w->cpl, (size_t)nwk * 4 * 8));
        CK(dalloc(A, &w->cpdet, (size_t)nwk * 8));
        CK(dalloc(A, &w->cpla, (size_t)nwk * 2 * 8));
        CK(dalloc(A, &w->cpsg, (size_t)nwk * 8));
        CK(dalloc(A, &w->cpsref, (size_t)nwk * 8));
        CK(dalloc(A, &w->cptmp, (size_t)nwk * (2 * fs + 2 * (size_t)ns * ns + 2) * 8));
    }
    // U_L = P^T for every walker and spin; U_R = phi0 (or P)
    std::vector<double> ul((size_t)nwk * 2 * fs), ur((size_t)nwk * 2 * fs);
    for (int j = 0; j < nwk; ++j)
        for (int sp = 0; sp < 2; ++sp) {
            double* l = ul.data() + ((size_t)j * 2 + sp) * fs;
            double* r = ur.data() + ((size_t)j * 2 + sp) * fs;
            const double* src = phi0 ? phi0 + ((size_t)w->gid[j] * 2 + sp) * fs : P;
            for (int i = 0; i < N; ++i)
                for (int c = 0; c < ns; ++c) {
                    l[(size_t)c * N + i] = P[(size_t)i * ns + c];
                    r[(size_t)i * ns + c] = src[(size_t)i * ns + c];
                }
        }
    CK(cudaMemcpyAsync(w->TUL, ul.data(), ul.size() * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w->TUR, ur.data(), ur.size() * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(w->cpl, 0, (size_t)nwk * 4 * 8, st));
    CK(cudaMemsetAsync(w->cpdet, 0, (size_t)nwk * 8, st));
    rc = cp_refresh(ctx, w, st, 1);
    if (rc) return rc;
    CK(cudaStreamSynchronize(st));  // the host staging goes out of scope
    rc = read_dev_err(ctx, w);
    if (rc) return rc;
    w->cp_logw.assign(nwk, 0.0);
    w->cp = true;
    w->gvalid = false;
    return AFQMC_OK;
}

int afqmc_cp_step(afqmc_ctx* ctx, int mode, int k, int nb, double* logw_step, void* stream) {
    int rc = cp_check(ctx, true);
    if (rc) return rc;
    const int NW = window_max<double>();
    if (mode == AFQMC_MODE_LOCAL) k = 1;
    else if (mode == AFQMC_MODE_BLOCKFB && (nb < 1 || nb > 32)) return AFQMC_ERR_ARG;
    else if (mode == AFQMC_MODE_DELAYED && (k < 1 || k > NW)) return AFQMC_ERR_ARG;
    else if (mode != AFQMC_MODE_DELAYED && mode != AFQMC_MODE_BLOCKFB) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    Walker* w = ctx->w[0];
    const int N = w->N, ns = w->nsm, nwk = w->nwk;
    const long fs = (long)N * ns, os = (long)ns * ns;
    w->gvalid = false;
    {
        PhaseScope ps(ctx, AFQMC_PHASE_PREP, st);
        CK(launch_uniforms(st, ctx->p.seed, w->gid_d, w->visit_d, 2 * N, w->u, nwk));
        CK(cudaMemsetAsync(w->stats, 0, (size_t)nwk * 8 * sizeof(int), st));
        CK(cudaMemsetAsync(w->maxr, 0, (size_t)nwk * 8, st));
    }
    {  // e^{-dtau K} phi: the separable passes over the site index of U_R (N x n_s)
        PhaseScope ps(ctx, AFQMC_PHASE_WRAP, st);
        SepArgs r;
        r.G = w->TUR; r.ld = ns; r.sG = fs;
        r.L = w->L; r.N = N; r.C = ns; r.batch = 2 * nwk; r.side = 0;
        r.A = w->lat->Ex64; r.circ = 1; r.sv = N; r.w = ctx->sep_tile;
        CK(launch_sep<double>(st, r));
    }
    {
        PhaseScope ps(ctx, AFQMC_PHASE_RECOMPUTE, st);
        rc = cp_refresh(ctx, w, st, 0);
        if (rc) return rc;
    }
    SiteParams sp;
    sp.N = N;
    sp.ld = w->ld;
    sp.c[0] = ctx->c[0];
    sp.c[1] = ctx->c[1];
    sp.lam = ctx->lam;
    sp.hs = ctx->p.hs;
    sp.seed = ctx->p.seed;
    sp.walker = (uint64_t)w->gid[0];
    sp.visit = w->visit;
    for (int s = 0; s < 2; ++s)
        for (int xi = 0; xi < 2; ++xi) {
            const double x = xi == 0 ? 1.0 : -1.0;
            sp.dflip[s][xi] = exp(ctx->c[s] * x) - 1.0;  // the field set from none
            sp.dstrip[s][xi] = 0.0;
        }
    for (int xi = 0; xi < 2; ++xi) {
        const double x = xi == 0 ? 1.0 : -1.0;
        sp.sflip[xi] = 0.5 * ((ctx->p.hs == AFQMC_HS_CHARGE_REAL) ? exp(-ctx->lam * x) : 1.0);  // p(x) s(x)
    }
    rc = tform_windows<double>(ctx, w, st, w->x, mode == AFQMC_MODE_BLOCKFB ? WIN_MODE_CPB : WIN_MODE_CP, k, nb, sp,
                               nullptr, w->cpl, 1.0);
    if (rc) return rc;
    count_launch();
    cp_finish_kernel<<<(nwk + 127) / 128, 128, 0, st>>>(w->cpl, w->cpdet, w->acc2, nwk);
    CK(cudaGetLastError());
    CK(launch_bump(st, w->visit_d));
    w->visit++;
    CK(cudaStreamSynchronize(st));
    rc = read_dev_err(ctx, w);
    if (rc) return rc;
    std::vector<double> h(nwk);
    CK(cudaMemcpy(h.data(), w->acc2, (size_t)nwk * 8, cudaMemcpyDeviceToHost));
    int src = -1;
    for (int j = 0; j < nwk; ++j) {
        w->cp_logw[j] += h[j];
        if (logw_step) logw_step[w->gid[j]] = h[j];
        if (src < 0 && std::isfinite(w->cp_logw[j])) src = j;
    }
    if (src < 0) return AFQMC_ERR_NUMERIC;  // every walker removed
    // a removed walker keeps weight zero; its slot takes a copy of a live walker's basis so that its
    // matrices stay regular until the next population control drops it
    for (int j = 0; j < nwk; ++j) {
        if (std::isfinite(w->cp_logw[j])) continue;
        for (int sp2 = 0; sp2 < 2; ++sp2) {
            CK(cudaMemcpyAsync((double*)w->TUR + ((size_t)j * 2 + sp2) * fs,
                               (const double*)w->TUR + ((size_t)src * 2 + sp2) * fs, fs * 8,
                               cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync((double*)w->TT + ((size_t)j * 2 + sp2) * os,
                               (const double*)w->TT + ((size_t)src * 2 + sp2) * os, os * 8,
                               cudaMemcpyDeviceToDevice, st));
        }
        CK(cudaMemcpyAsync(w->cpdet + j, w->cpdet + src, 8, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(w->cpsref + j, w->cpsref + src, 8, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemsetAsync(w->cpl + 4 * j + 2, 0, 8, st));
    }
    return AFQMC_OK;
}

int afqmc_cp_comb(afqmc_ctx* ctx, double u0, int* idx_out, void* stream) {
    int rc = cp_check(ctx, true);
    if (rc) return rc;
    if (!(u0 >= 0.0 && u0 < 1.0)) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    Walker* w = ctx->w[0];
    const int nwk = w->nwk, N = w->N, ns = w->nsm;
    const long fs = (long)N * ns, os = (long)ns * ns;
    double mx = -INFINITY;
    for (double v : w->cp_logw) mx = std::max(mx, v);
    if (!std::isfinite(mx)) return AFQMC_ERR_NUMERIC;
    std::vector<double> cum(nwk);
    double tot = 0.0;
    for (int j = 0; j < nwk; ++j) {
        tot += std::isfinite(w->cp_logw[j]) ? exp(w->cp_logw[j] - mx) : 0.0;
        cum[j] = tot;
    }
    std::vector<int> idx(nwk);
    for (int q = 0; q < nwk; ++q) {
        const double pos = (q + u0) * tot / nwk;
        int j = (int)(std::upper_bound(cum.begin(), cum.end(), pos) - cum.begin());
        idx[q] = std::min(j, nwk - 1);
    }
    double* tmp = w->cptmp;  // gather through scratch
    const long per = 2 * fs + 2 * os + 2;
    for (int q = 0; q < nwk; ++q) {
        const int j = idx[q];
        double* t = tmp + (size_t)q * per;
        CK(cudaMemcpyAsync(t, (const double*)w->TUR + (size_t)j * 2 * fs, 2 * fs * 8, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(t + 2 * fs, (const double*)w->TT + (size_t)j * 2 * os, 2 * os * 8, cudaMemcpyDeviceToDevice,
                           st));
        CK(cudaMemcpyAsync(t + 2 * fs + 2 * os, w->cpdet + j, 8, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(t + 2 * fs + 2 * os + 1, w->cpsref + j, 8, cudaMemcpyDeviceToDevice, st));
    }
    for (int q = 0; q < nwk; ++q) {
        const double* t = tmp + (size_t)q * per;
        CK(cudaMemcpyAsync((double*)w->TUR + (size_t)q * 2 * fs, t, 2 * fs * 8, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync((double*)w->TT + (size_t)q * 2 * os, t + 2 * fs, 2 * os * 8, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(w->cpdet + q, t + 2 * fs + 2 * os, 8, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(w->cpsref + q, t + 2 * fs + 2 * os + 1, 8, cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaMemsetAsync(w->cpl, 0, (size_t)nwk * 4 * 8, st));
    const double lw = mx + log(tot / nwk);
    for (int q = 0; q < nwk; ++q) w->cp_logw[q] = lw;
    w->gvalid = false;
    if (idx_out)
        for (int q = 0; q < nwk; ++q) idx_out[q] = w->gid[idx[q]];
    CK(cudaStreamSynchronize(st));
    return read_dev_err(ctx, w);
}

int afqmc_cp_reorth(afqmc_ctx* ctx, void* stream) {
    int rc = cp_check(ctx, true);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    Walker* w = ctx->w[0];
    const Fac R{(double*)w->TUR, 2 * (long)w->N * w->nsm, (long)w->N * w->nsm};
    CK(stab_rows(ctx, w, st, R, 0, 2, nullptr));
    rc = cp_refresh(ctx, w, st, 1);
    if (rc) return rc;
    w->gvalid = false;
    CK(cudaStreamSynchronize(st));
    return read_dev_err(ctx, w);
}

int afqmc_cp_energy(afqmc_ctx* ctx, double* e_local, double* e_mean, void* stream) {
    int rc = cp_check(ctx, true);
    if (rc) return rc;
    if (!e_local && !e_mean) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    Walker* w = ctx->w[0];
    CK(tform_form_G<double>(w, st));  // the mixed G = 1 - U_R T U_L
    CK(cudaMemsetAsync(w->acc2, 0, (size_t)w->nwk * 16, st));
    CK(launch_energy<double>(st, (const double*)w->G, w->ld, w->L, ctx->p.t, ctx->p.U, w->acc2, w->nwk,
                             w->gstride()));
    CK(cudaStreamSynchronize(st));
    rc = read_dev_err(ctx, w);
    if (rc) return rc;
    std::vector<double> e(w->nwk);
    CK(cudaMemcpy(e.data(), w->acc2, (size_t)w->nwk * 8, cudaMemcpyDeviceToHost));
    double mx = -INFINITY, num = 0.0, den = 0.0;
    for (double v : w->cp_logw) mx = std::max(mx, v);
    for (int j = 0; j < w->nwk; ++j) {
        if (e_local) e_local[w->gid[j]] = e[j];
        const double wt = std::isfinite(w->cp_logw[j]) ? exp(w->cp_logw[j] - mx) : 0.0;
        num += wt * e[j];
        den += wt;
    }
    if (e_mean) *e_mean = den > 0.0 ? num / den : NAN;
    return AFQMC_OK;
}

int afqmc_cp_get_walker(afqmc_ctx* ctx, int walker, double* phi, double* logw) {
    int rc = cp_check(ctx, true);
    if (rc) return rc;
    if (walker < 0 || walker >= (int)ctx->wmap.size()) return AFQMC_ERR_ARG;
    Walker* w = ctx->w[ctx->wmap[walker].first];
    const int j = ctx->wmap[walker].second;
    if (ctx->last) CK(cudaStreamSynchronize(ctx->last));
    const size_t fs = (size_t)w->N * w->nsm;
    if (phi) CK(cudaMemcpy(phi, (const double*)w->TUR + (size_t)j * 2 * fs, 2 * fs * 8, cudaMemcpyDeviceToHost));
    if (logw) *logw = w->cp_logw[j];
    return AFQMC_OK;
}

int afqmc_measure_energy(afqmc_ctx* ctx, double* energy, double* sign, void* stream) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (ctx->w.empty() || !energy) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    for (auto* w : ctx->w) {
        if (!w->gvalid) {
            if (ctx->p.precision == AFQMC_PREC_FP64) CK(tform_form_G<double>(w, st));
            else CK(tform_form_G<float>(w, st));
        }
        CK(cudaMemsetAsync(w->acc2, 0, (size_t)w->nwk * 16, st));
        if (ctx->p.precision == AFQMC_PREC_FP64)
            CK(launch_energy<double>(st, (const double*)w->G, w->ld, w->L, ctx->p.t, ctx->p.U, w->acc2, w->nwk,
                                     w->gstride()));
        else
            CK(launch_energy<float>(st, (const float*)w->G, w->ld, w->L, ctx->p.t, ctx->p.U, w->acc2, w->nwk,
                                    w->gstride()));
    }
    CK(cudaStreamSynchronize(st));
    for (auto* w : ctx->w) {
        int r = read_dev_err(ctx, w);
        if (r) return r;
        std::vector<double> e(w->nwk), sg(w->nwk);
        CK(cudaMemcpy(e.data(), w->acc2, (size_t)w->nwk * 8, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(sg.data(), w->sign, (size_t)w->nwk * 8, cudaMemcpyDeviceToHost));
        for (int j = 0; j < w->nwk; ++j) {
            energy[w->gid[j]] = e[j];
            if (sign) sign[w->gid[j]] = sg[j];
        }
    }
    return AFQMC_OK;
}

static bool walker_of(afqmc_ctx* ctx, int walker, Walker** w, int* j) {
    if (!ctx || walker < 0 || walker >= (int)ctx->wmap.size()) return false;
    *w = ctx->w[ctx->wmap[walker].first];
    *j = ctx->wmap[walker].second;
    return true;
}

int afqmc_get_G(afqmc_ctx* ctx, int walker, int spin, double* host_out) {
    Walker* w;
    int j;
    if (!walker_of(ctx, walker, &w, &j) || spin < 0 || spin > 1 || !host_out) return AFQMC_ERR_ARG;
    if (!w->gvalid) {  // T form: G = 1 - U_R T U_L on the stream of the last call
        if (ctx->p.precision == AFQMC_PREC_FP64) CK(tform_form_G<double>(w, ctx->last));
        else CK(tform_form_G<float>(w, ctx->last));
    }
    CK(cudaStreamSynchronize(ctx->last));
    const size_t es = esize(ctx);
    std::vector<char> buf((size_t)w->N * w->ld * es);
    CK(cudaMemcpy(buf.data(), (char*)w->G + ((size_t)j * 2 + spin) * w->N * w->ld * es, buf.size(),
                  cudaMemcpyDeviceToHost));
    for (int i = 0; i < w->N; ++i)
        for (int c = 0; c < w->N; ++c) {
            size_t o = (size_t)i * w->ld + c;
            host_out[(size_t)i * w->N + c] = (es == 8) ? ((double*)buf.data())[o] : (double)((float*)buf.data())[o];
        }
    return read_dev_err(ctx, w);
}

int afqmc_set_G(afqmc_ctx* ctx, int walker, int spin, const double* host_in) {
    Walker* w;
    int j;
    if (!walker_of(ctx, walker, &w, &j) || spin < 0 || spin > 1 || !host_in) return AFQMC_ERR_ARG;
    if (ctx->form == AFQMC_FORM_T) return AFQMC_ERR_STATE;  // the T form's state is not G
    CK(cudaStreamSynchronize(ctx->last));
    const size_t es = esize(ctx);
    std::vector<char> buf((size_t)w->N * w->ld * es, 0);
    for (int i = 0; i < w->N; ++i)
        for (int c = 0; c < w->N; ++c) {
            size_t o = (size_t)i * w->ld + c;
            double v = host_in[(size_t)i * w->N + c];
            if (es == 8) ((double*)buf.data())[o] = v;
            else ((float*)buf.data())[o] = (float)v;
        }
    CK(cudaMemcpy((char*)w->G + ((size_t)j * 2 + spin) * w->N * w->ld * es, buf.data(), buf.size(),
                  cudaMemcpyHostToDevice));
    return AFQMC_OK;
}

int afqmc_get_fields(afqmc_ctx* ctx, int walker, int8_t* host_out) {
    Walker* w;
    int j;
    if (!walker_of(ctx, walker, &w, &j) || !host_out) return AFQMC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->last));
    CK(cudaMemcpy(host_out, w->x + (size_t)j * ctx->p.M * w->N, (size_t)ctx->p.M * w->N, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

int afqmc_get_decisions(afqmc_ctx* ctx, int walker, uint8_t* host_out) {
    Walker* w;
    int j;
    if (!walker_of(ctx, walker, &w, &j) || !host_out) return AFQMC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->last));
    CK(cudaMemcpy(host_out, w->dec + (size_t)j * 2 * w->N, 2 * (size_t)w->N, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

int afqmc_get_ratios(afqmc_ctx* ctx, int walker, double* host_out) {
    Walker* w;
    int j;
    if (!walker_of(ctx, walker, &w, &j) || !host_out) return AFQMC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->last));
    CK(cudaMemcpy(host_out, w->ratio + (size_t)j * 2 * w->N, 2 * (size_t)w->N * 8, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

int afqmc_get_info(afqmc_ctx* ctx, int walker, int* N, int* n_up, int* n_dn, int* slice, int* dir) {
    Walker* w;
    int j;
    if (!walker_of(ctx, walker, &w, &j)) return AFQMC_ERR_ARG;
    if (N) *N = w->N;
    if (n_up) *n_up = w->ns[0];
    if (n_dn) *n_dn = w->ns[1];
    if (slice) *slice = w->pos;
    if (dir) *dir = w->last_dir;
    return AFQMC_OK;
}

int afqmc_set_graphs(afqmc_ctx* ctx, int on) {
    if (!ctx) return AFQMC_ERR_ARG;
    ctx->graphs = on != 0;
    return AFQMC_OK;
}

int afqmc_set_wrap(afqmc_ctx* ctx, int mode) {
    if (!ctx || (mode != AFQMC_WRAP_DENSE && mode != AFQMC_WRAP_SEPARABLE)) return AFQMC_ERR_ARG;
    if (mode == AFQMC_WRAP_SEPARABLE) {
        for (auto* w : ctx->w) {
            const bool ok = ctx->p.precision == AFQMC_PREC_FP64 ? sep_available<double>(w->L, w->N) : sep_available<float>(w->L, w->N);
            if (!ok) return AFQMC_ERR_ARG;
        }
    }
    ctx->wrap_mode = mode;
    return AFQMC_OK;
}

int afqmc_set_form(afqmc_ctx* ctx, int form) {
    if (!ctx || (form != AFQMC_FORM_G && form != AFQMC_FORM_T)) return AFQMC_ERR_ARG;
    if (!ctx->w.empty()) return AFQMC_ERR_STATE;
    ctx->form = form;
    return AFQMC_OK;
}

int afqmc_set_wrap_tile(afqmc_ctx* ctx, int width) {
    if (!ctx || width < 0) return AFQMC_ERR_ARG;
    if (width > 0)
        for (auto* w : ctx->w) {
            const bool ok = ctx->p.precision == AFQMC_PREC_FP64 ? sep_width_fits<double>(w->L, w->N, width)
                                                                : sep_width_fits<float>(w->L, w->N, width);
            if (!ok) return AFQMC_ERR_ARG;
        }
    ctx->sep_tile = width;
    return AFQMC_OK;
}

// Wait for every stream a phase interval may sit on: the caller's last stream and each group's
// main, flush and propagation streams (the recompute's deferred re-orthonormalisation runs on
// the last).
static cudaError_t sync_profiled_streams(afqmc_ctx* ctx) {
    cudaError_t e = cudaSuccess;
    if (ctx->last && (e = cudaStreamSynchronize(ctx->last)) != cudaSuccess) return e;
    for (auto* w : ctx->w)
        for (cudaStream_t q : {w->sm, w->sf, w->sp})
            if (q && (e = cudaStreamSynchronize(q)) != cudaSuccess) return e;
    return cudaSuccess;
}

int afqmc_set_profiling(afqmc_ctx* ctx, int on) {
    if (!ctx) return AFQMC_ERR_ARG;
    CK(sync_profiled_streams(ctx));
    for (auto& pe : ctx->prof.pending) {
        ctx->prof.pool.push_back(pe.a);
        ctx->prof.pool.push_back(pe.b);
    }
    ctx->prof.pending.clear();
    for (int i = 0; i < AFQMC_NPHASE; ++i) {
        ctx->prof.ms[i] = 0.0;
        ctx->prof.intervals[i] = 0;
        ctx->prof.launches[i] = 0;
    }
    ctx->prof.on = on != 0;
    return AFQMC_OK;
}

int afqmc_get_profile(afqmc_ctx* ctx, double* ms, int64_t* intervals, int64_t* launches) {
    if (!ctx) return AFQMC_ERR_ARG;
    CK(sync_profiled_streams(ctx));
    // an interval leaves the pending list as its events return to the pool, so an error part way
    // leaves each event in exactly one of the two lists (both are destroyed with the context)
    while (!ctx->prof.pending.empty()) {
        const auto pe = ctx->prof.pending.back();
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, pe.a, pe.b));
        ctx->prof.ms[pe.phase] += t;
        ctx->prof.intervals[pe.phase] += 1;
        ctx->prof.pending.pop_back();
        ctx->prof.pool.push_back(pe.a);
        ctx->prof.pool.push_back(pe.b);
    }
    for (int i = 0; i < AFQMC_NPHASE; ++i) {
        if (ms) ms[i] = ctx->prof.ms[i];
        if (intervals) intervals[i] = ctx->prof.intervals[i];
        if (launches) launches[i] = ctx->prof.launches[i];
    }
    return AFQMC_OK;
}

int64_t afqmc_launch_count(void) { return (int64_t)g_launches.load(); }

int afqmc_debug_gemm(int kind, int M, int N, int K, const float* A, long long lda, const float* Bt, long long ldb,
                     float* C, long long ldc, int c_trans, void* stream) {
    if ((kind != 1 && kind != 2) || M < 1 || N < 1 || K < 1 || !A || !Bt || !C) return AFQMC_ERR_ARG;
    if (lda < K || ldb < K || ldc < (c_trans ? M : N)) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int* err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return AFQMC_ERR_OOM;
    cudaMemsetAsync(err, 0, sizeof(int), st);
    TcGemmArgs g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda;
    g.Bt = Bt; g.ldb = ldb;
    g.C = C; g.ldc = ldc; g.c_trans = c_trans;
    g.split3 = kind == 2;
    g.err = err;
    cudaError_t e = tc_gemm(st, g);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(err);
    if (e == cudaErrorInvalidValue) return AFQMC_ERR_ARG;  // a tensor map refused the pointers or strides
    if (e != cudaSuccess) return AFQMC_ERR_CUDA;
    if (h == DEV_TIMEOUT) return AFQMC_ERR_TIMEOUT;
    return h ? AFQMC_ERR_CUDA : AFQMC_OK;
}

int afqmc_debug_dgemm(int kind, int M, int N, int K, const double* A, long long lda, const double* B, long long ldb,
                      double* C, long long ldc, void* stream) {
    if ((kind != 0 && kind != 1) || M < 1 || N < 1 || K < 1 || !A || !B || !C) return AFQMC_ERR_ARG;
    if (lda < K || ldb < N || ldc < N) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int* err = nullptr;
    void* ws = nullptr;
    double* sc = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return AFQMC_ERR_OOM;
    if (kind == 1 && (cudaMalloc(&ws, ozaki_ws_bytes(M, N, K, 1)) != cudaSuccess ||
                      cudaMalloc(&sc, ozaki_sc_doubles(M, N, 1) * sizeof(double)) != cudaSuccess)) {
        cudaFree(ws);
        cudaFree(err);
        return AFQMC_ERR_OOM;
    }
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess && kind == 0) {
        GemmArgs<double> g;
        g.M = M; g.N = N; g.K = K;
        g.A = A; g.lda = lda;
        g.B = B; g.ldb = ldb;
        g.C = C; g.ldc = ldc;
        e = gemm<double>(st, g);
    } else if (e == cudaSuccess) {
        OzGemmArgs o;
        o.M = M; o.N = N; o.K = K;
        o.A = A; o.lda = lda;
        o.B = B; o.ldb = ldb;
        o.C = C; o.ldc = ldc;
        o.err = err;
        e = ozaki_gemm(st, o, ws, sc);
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(sc);
    cudaFree(ws);
    cudaFree(err);
    if (e == cudaErrorInvalidValue) return AFQMC_ERR_ARG;
    if (e != cudaSuccess) return AFQMC_ERR_CUDA;
    if (h == DEV_TIMEOUT) return AFQMC_ERR_TIMEOUT;
    if (h == DEV_NUMERIC) return AFQMC_ERR_NUMERIC;
    return h ? AFQMC_ERR_CUDA : AFQMC_OK;
}

int afqmc_debug_ozaki_plan(int M, int N, int K, int batch, int* b, int* s, int* ngroups, int cap, int* np, int* pa,
                           int* pb) {
    if (!b || !s || !ngroups || cap < 0 || (cap > 0 && (!np || !pa || !pb))) return AFQMC_ERR_ARG;
    return ozaki_plan_info(M, N, K, batch, b, s, ngroups, cap, np, pa, pb) == 0 ? AFQMC_OK : AFQMC_ERR_ARG;
}

int afqmc_debug_wait_timeout(long long limit_ns, void* stream) {
    if (limit_ns < 1000 || limit_ns > 2000000000LL) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int* buf = nullptr;  // [0] the error word, [1] the flag that nothing sets
    if (cudaMalloc(&buf, 2 * sizeof(int)) != cudaSuccess) return AFQMC_ERR_OOM;
    cudaError_t e = cudaMemsetAsync(buf, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) {
        count_launch();
        debug_wait_kernel<<<1, 32, 0, st>>>((const unsigned int*)(buf + 1), (unsigned long long)limit_ns, buf);
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, buf, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) return AFQMC_ERR_CUDA;
    if (h == DEV_TIMEOUT) return AFQMC_ERR_TIMEOUT;
    return h ? AFQMC_ERR_CUDA : AFQMC_OK;
}

int afqmc_debug_uniforms(uint64_t seed, uint64_t walker, uint64_t visit, int count, double* host_out) {
    if (count < 0 || (count > 0 && !host_out)) return AFQMC_ERR_ARG;
    if (count == 0) return AFQMC_OK;
    double* d = nullptr;
    if (cudaMalloc(&d, (size_t)count * 8) != cudaSuccess) return AFQMC_ERR_OOM;
    count_launch();
    debug_uniforms_kernel<<<(count + 255) / 256, 256>>>(seed, walker, visit, count, d);
    cudaError_t e = cudaMemcpy(host_out, d, (size_t)count * 8, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? AFQMC_OK : AFQMC_ERR_CUDA;
}

}  // extern "C"
