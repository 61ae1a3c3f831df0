// abi.cu -- the C ABI of libafqmc.so (include/afqmc.h): contexts, walkers and
// the orchestration of one slice of the PQMC sweep (Sec. II.B-II.D, III).
#include <math.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "internal.h"

namespace afq {
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches += n; }
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
    double* Ex64 = nullptr;  // L x L: exp(-dtau K) = Ex (x) Ex for the periodic square lattice
};

struct Walker {
    int L = 0, N = 0;
    long ld = 0;
    int ns[2] = {0, 0};
    int pos = 0, last_dir = -1;
    bool need_recompute = false;
    uint64_t visit = 0;
    Lattice* lat = nullptr;
    void* G = nullptr;      // [2][N][ld] bulk
    void* Tbuf = nullptr;   // [2][N][ld] bulk (wrap temporary)
    int8_t* x = nullptr;    // M x N
    double* u = nullptr;    // 2N uniforms
    void* dvec = nullptr;   // bulk [2][N] d, then [2][N] dinv
    double* d64 = nullptr;  // FP64 [2][N] d, [2][N] dinv
    uint8_t* dec = nullptr;
    double* ratio = nullptr;
    int* stats = nullptr;   // 4 ints
    double* maxr = nullptr;
    double* sign = nullptr;
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
    cudaEvent_t ev_chain[2] = {nullptr, nullptr}, ev_prod[2] = {nullptr, nullptr}, ev_done = nullptr;
    double* URs[2] = {nullptr, nullptr};
    double* ULs[2] = {nullptr, nullptr};
    int nsm = 0;                 // max(ns[0], ns[1])
    double* Ucur = nullptr;      // 2 x N x nsm: the factor being propagated, per spin
    double* Utmp = nullptr;      // N x nsm: propagation scratch
    double* Ut2 = nullptr;       // 2 x N x nsm: transposed left factors for the LU
    double* Ob = nullptr;        // 2 x nsm x nsm: U_L U_R, then its LU
    double* Z = nullptr;         // 2 x nsm x N: (U_L U_R)^{-1} U_L
    double* Gnew = nullptr;      // N x ld: the recomputed G of one spin
    int* perm2 = nullptr;        // 2 x max(N, nsm): pivot rows
    int8_t* flag2 = nullptr;     // 2 x max(N, nsm): pivoted-row flags
    int* visited = nullptr;      // max(N, nsm): permutation-parity scratch
    double* acc2 = nullptr;
    std::vector<void*> allocs;
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
    std::vector<Lattice*> lats;
    std::vector<Walker*> w;
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
__global__ void transpose_kernel(const double* A, int rows, int cols, double* B) {  // B = A^T
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)rows * cols; e += (long)gridDim.x * blockDim.x) {
        int r = (int)(e / cols), c = (int)(e % cols);
        B[(long)c * rows + r] = A[e];
    }
}

__global__ void fields_kernel(uint64_t seed, uint64_t walker, long count, int8_t* x) {
    long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count) x[j] = philox_uniform(seed, walker, ~0ULL, (uint64_t)j) < 0.5 ? 1 : -1;
}

__global__ void set_double_kernel(double* p, double v) { *p = v; }

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

static Lattice* get_lattice(afqmc_ctx* ctx, int L, cudaStream_t st, cudaError_t* err) {
    for (auto* l : ctx->lats)
        if (l->L == L) return l;
    Lattice* l = new Lattice();
    l->L = L;
    l->N = L * L;
    l->ld = ((l->N + 31) / 32) * 32;
    size_t n2 = (size_t)l->N * l->ld;
    *err = cudaSuccess;
    if ((*err = dalloc(ctx->allocs, &l->E64, n2 * 8)) != cudaSuccess) return nullptr;
    if ((*err = dalloc(ctx->allocs, &l->Einv64, n2 * 8)) != cudaSuccess) return nullptr;
    if ((*err = dalloc(ctx->allocs, (char**)&l->Eb, n2 * esize(ctx))) != cudaSuccess) return nullptr;
    if ((*err = dalloc(ctx->allocs, (char**)&l->Einvb, n2 * esize(ctx))) != cudaSuccess) return nullptr;
    if ((*err = dalloc(ctx->allocs, &l->Ex64, (size_t)L * L * 8)) != cudaSuccess) return nullptr;
    if ((*err = launch_expK1d(st, L, ctx->p.t, ctx->p.dtau, l->Ex64)) != cudaSuccess) return nullptr;
    if ((*err = launch_expK(st, L, ctx->p.t, ctx->p.dtau, l->E64, l->ld)) != cudaSuccess) return nullptr;
    if ((*err = launch_expK(st, L, ctx->p.t, -ctx->p.dtau, l->Einv64, l->ld)) != cudaSuccess) return nullptr;
    if (ctx->p.precision == AFQMC_PREC_FP64) {
        if ((*err = launch_cast<double>(st, l->E64, l->ld, (double*)l->Eb, l->ld, l->N, l->N)) != cudaSuccess) return nullptr;
        if ((*err = launch_cast<double>(st, l->Einv64, l->ld, (double*)l->Einvb, l->ld, l->N, l->N)) != cudaSuccess) return nullptr;
    } else {
        if ((*err = launch_cast<float>(st, l->E64, l->ld, (float*)l->Eb, l->ld, l->N, l->N)) != cudaSuccess) return nullptr;
        if ((*err = launch_cast<float>(st, l->Einv64, l->ld, (float*)l->Einvb, l->ld, l->N, l->N)) != cudaSuccess) return nullptr;
    }
    ctx->lats.push_back(l);
    return l;
}

static cudaError_t prop_right(afqmc_ctx* ctx, Walker* w, cudaStream_t st, int s, int ell, double* U, double* tmp);
static cudaError_t prop_left(afqmc_ctx* ctx, Walker* w, cudaStream_t st, int s, int ell, double* U, double* tmp);
// Propagate both spins' factors U[s] over nsl slices l = l_first, l_first + l_step, ...
// (right factors N x ns: B_l U; left factors ns x N: U B_l) with the fused kernel; lattices too
// large for it take the per-slice separable products.
static cudaError_t propagate(afqmc_ctx* ctx, Walker* w, cudaStream_t st, double* const* U, int left, int l_first,
                             int l_step, int nsl) {
    const int N = w->N;
    PropArgs a;
    for (int s = 0; s < 2; ++s) {
        a.U[s] = U[s];
        a.nvec[s] = w->ns[s];
        a.vs[s] = left ? N : 1;
        a.es[s] = left ? 1 : w->ns[s];
        a.dplus[s] = exp(ctx->c[s]);
        a.dminus[s] = exp(-ctx->c[s]);
    }
    a.Ex = w->lat->Ex64;
    a.x = w->x;
    a.L = w->L;
    a.l_first = l_first;
    a.l_step = l_step;
    a.nsl = nsl;
    a.left = left;
    a.nmat = 2;
    cudaError_t e = launch_prop(st, a);
    if (e != cudaErrorInvalidValue) return e;
    cudaGetLastError();
    for (int t = 0; t < nsl; ++t)
        for (int s = 0; s < 2; ++s) {
            const int ell = l_first + t * l_step;
            e = left ? prop_left(ctx, w, st, s, ell, U[s], w->Utmp) : prop_right(ctx, w, st, s, ell, U[s], w->Utmp);
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

static LuArgs lu_args(Walker* w, double* const* A, int nmat, long lda, int m, int n) {
    const int maxr = w->N > w->nsm ? w->N : w->nsm;
    LuArgs a;
    for (int q = 0; q < nmat; ++q) {
        a.A[q] = A[q];
        a.perm[q] = w->perm2 + (size_t)q * maxr;
        a.flag[q] = w->flag2 + (size_t)q * maxr;
    }
    a.lda = lda;
    a.m = m;
    a.n = n;
    a.nmat = nmat;
    a.err = w->err;
    return a;
}

// Re-orthonormalisation (Sec. II.C): every U[q] (N x ns, row-major) becomes P L from its
// partially pivoted LU, a basis of the same column space with entries of magnitude <= 1 (only
// the column space enters G, Eq. GrFMatNew).  *sign (nullable) is multiplied by the sign of the
// discarded triangular factor.
static cudaError_t stab_rows(afqmc_ctx* ctx, Walker* w, cudaStream_t st, double* const* U, int nmat, int ns,
                             double* sign) {
    LuArgs a = lu_args(w, U, nmat, ns, w->N, ns);
    cudaError_t e;
    {
        PhaseScope ps(ctx, AFQMC_PHASE_ELIM, st);
        if ((e = launch_lu(st, a)) != cudaSuccess) return e;
    }
    if (sign && (e = launch_lu_sign(st, a, 0, sign, w->visited)) != cudaSuccess) return e;
    return launch_lu_unit_rows(st, a);
}

// The same for left factors U[q] (ns x N): through their transposes.
static cudaError_t stab_cols(afqmc_ctx* ctx, Walker* w, cudaStream_t st, double* const* U, int nmat, int ns,
                             double* sign) {
    const int N = w->N;
    double* T[2] = {w->Ut2, w->Ut2 + (size_t)N * w->nsm};
    cudaError_t e;
    for (int q = 0; q < nmat; ++q) {
        count_launch();
        transpose_kernel<<<256, 256, 0, st>>>(U[q], ns, N, T[q]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = stab_rows(ctx, w, st, T, nmat, ns, sign)) != cudaSuccess) return e;
    for (int q = 0; q < nmat; ++q) {
        count_launch();
        transpose_kernel<<<256, 256, 0, st>>>(T[q], N, ns, U[q]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Z[q] = (UL[q] UR[q])^{-1} UL[q] (ns x N) for the spins of a group (Eq. GrFMatNew):
// O = UL UR (FP64), its pivoted LU, then the substitutions with UL as right-hand side.
// *sign (nullable) is multiplied by sign(det O) of every spin.
static cudaError_t form_Z(afqmc_ctx* ctx, Walker* w, cudaStream_t st, const double* const* UR, const double* const* UL,
                          int nmat, int ns, double* sign) {
    const int N = w->N;
    double* O[2] = {w->Ob, w->Ob + (size_t)w->nsm * w->nsm};
    double* Z[2] = {w->Z, w->Z + (size_t)w->nsm * N};
    cudaError_t e;
    for (int q = 0; q < nmat; ++q) {
        GemmArgs<double> g;
        g.M = ns; g.N = ns; g.K = N;
        g.A = UL[q]; g.lda = N;
        g.B = UR[q]; g.ldb = ns;
        g.C = O[q]; g.ldc = ns;
        if ((e = gemm<double>(st, g)) != cudaSuccess) return e;
    }
    LuArgs a = lu_args(w, O, nmat, ns, ns, ns);
    {
        PhaseScope ps(ctx, AFQMC_PHASE_LU_O, st);
        if ((e = launch_lu(st, a)) != cudaSuccess) return e;
    }
    if (sign && (e = launch_lu_sign(st, a, 1, sign, w->visited)) != cudaSuccess) return e;
    SolveArgs sa;
    for (int q = 0; q < nmat; ++q) {
        sa.LU[q] = O[q];
        sa.perm[q] = a.perm[q];
        sa.B[q] = UL[q];
        sa.Z[q] = Z[q];
    }
    sa.ldl = ns;
    sa.ns = ns;
    sa.N = N;
    sa.nmat = nmat;
    PhaseScope pv(ctx, AFQMC_PHASE_SOLVE, st);
    return launch_lu_solve(st, sa);
}

// G_new (FP64, N x ld) = 1 - UR Z for the spin whose Z sits at slot q of form_Z.  The N x N
// product stays in FP64 for both bulk precisions: the LU bases are not orthonormal, so 1 - UR Z
// cancels large terms and an FP32 product would lose the digits the recompute restores.
static cudaError_t finish_G(Walker* w, cudaStream_t st, const double* UR, int q, int ns) {
    const int N = w->N;
    GemmArgs<double> h;
    h.M = N; h.N = N; h.K = ns;
    h.A = UR; h.lda = ns;
    h.B = w->Z + (size_t)q * w->nsm * N; h.ldb = N;
    h.C = w->Gnew; h.ldc = w->ld;
    cudaError_t e = gemm<double>(st, h);
    if (e != cudaSuccess) return e;
    return launch_identity_minus<double>(st, w->Gnew, w->ld, N);
}

// U (N x ns) <- B_l U, B_l = diag(exp(c_s x_l)) E.  E = Ex (x) Ex on the square lattice, so
// E U is two small products: along x for every row block y, then along y.
static cudaError_t prop_right(afqmc_ctx* ctx, Walker* w, cudaStream_t st, int s, int ell, double* U, double* tmp) {
    const int N = w->N, ns = w->ns[s], L = w->L;
    cudaError_t e = launch_field_scales_T<double>(st, w->x + (size_t)(ell - 1) * N, N, ctx->c, w->d64, w->d64 + 2 * N, N);
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

// U (ns x N) <- U B_l = (U diag(exp(c_s x_l))) E, with the same separable product.
static cudaError_t prop_left(afqmc_ctx* ctx, Walker* w, cudaStream_t st, int s, int ell, double* U, double* tmp) {
    const int N = w->N, ns = w->ns[s], L = w->L;
    cudaError_t e = launch_field_scales_T<double>(st, w->x + (size_t)(ell - 1) * N, N, ctx->c, w->d64, w->d64 + 2 * N, N);
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

template <typename T>
static cudaError_t store_G(Walker* w, cudaStream_t st, int s) {
    T* G = (T*)w->G + (size_t)s * w->N * w->ld;
    return launch_cast<T>(st, w->Gnew, w->ld, G, w->ld, w->N, w->N);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
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
        if (w->sf) cudaStreamDestroy(w->sf);
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
    size_t poff = 0, foff = 0;
    for (int wi = 0; wi < n_walkers; ++wi) {
        if (L[wi] < 2 || L[wi] > 64) return AFQMC_ERR_ARG;
        int N = L[wi] * L[wi];
        if (n_up[wi] < 1 || n_up[wi] > N || n_dn[wi] < 1 || n_dn[wi] > N) return AFQMC_ERR_ARG;
    }
    for (int wi = 0; wi < n_walkers; ++wi) {
        Walker* w = new Walker();
        ctx->w.push_back(w);
        cudaError_t e;
        w->lat = get_lattice(ctx, L[wi], st, &e);
        if (!w->lat) return fail(ctx, e);
        w->L = L[wi];
        w->N = w->lat->N;
        w->ld = w->lat->ld;
        w->ns[0] = n_up[wi];
        w->ns[1] = n_dn[wi];
        const int N = w->N;
        const long ld = w->ld;
        const int nsm = w->ns[0] > w->ns[1] ? w->ns[0] : w->ns[1];
        const int NW = (ctx->p.precision == AFQMC_PREC_FP64) ? window_max<double>() : window_max<float>();
        auto& A = w->allocs;
        CK(dalloc(A, (char**)&w->G, 2 * (size_t)N * ld * es));
        CK(dalloc(A, (char**)&w->Tbuf, 2 * (size_t)N * ld * es));
        CK(dalloc(A, &w->x, (size_t)M * N));
        CK(dalloc(A, &w->u, 2 * (size_t)N * 8));
        CK(dalloc(A, (char**)&w->dvec, 4 * (size_t)N * es));
        CK(dalloc(A, &w->d64, 4 * (size_t)N * 8));
        CK(dalloc(A, &w->dec, 2 * (size_t)N));
        CK(dalloc(A, &w->ratio, 2 * (size_t)N * 8));
        CK(dalloc(A, &w->stats, 8 * sizeof(int)));
        CK(dalloc(A, &w->maxr, 8));
        CK(dalloc(A, &w->sign, 8));
        CK(dalloc(A, &w->replay, 2 * (size_t)N));
        CK(dalloc(A, (char**)&w->colbuf, 4 * (size_t)N * es));
        CK(dalloc(A, (char**)&w->rowbuf, 4 * (size_t)N * es));
        CK(dalloc(A, &w->bar, sizeof(GridBar)));
        CK(dalloc(A, &w->err, sizeof(int)));
        for (int q = 0; q < 2; ++q) {
            CK(dalloc(A, &w->wm[q], 2 * sizeof(int)));
            CK(dalloc(A, &w->widx[q], (size_t)NW * sizeof(int)));
            CK(dalloc(A, &w->wdtot[q], 2 * (size_t)NW * 8));
            CK(dalloc(A, (char**)&w->Wm[q], 2 * (size_t)NW * NW * es));
            CK(dalloc(A, (char**)&w->Wx[q], 2 * (size_t)NW * NW * es));
            CK(dalloc(A, (char**)&w->X[q], 2 * (size_t)N * NW * es));
            CK(dalloc(A, (char**)&w->Y[q], 4 * (size_t)NW * N * es));
            CK(dalloc(A, (char**)&w->snap[q], 2 * (size_t)NW * NW * es));
            CK(cudaEventCreateWithFlags(&w->ev_chain[q], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&w->ev_prod[q], cudaEventDisableTiming));
        }
        CK(cudaEventCreateWithFlags(&w->ev_done, cudaEventDisableTiming));
        {
            int lo = 0, hi = 0;
            CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            CK(cudaStreamCreateWithPriority(&w->sf, cudaStreamNonBlocking, lo));
        }
        for (int s = 0; s < 2; ++s) {
            CK(dalloc(A, &w->URs[s], (size_t)nst * N * w->ns[s] * 8));
            CK(dalloc(A, &w->ULs[s], (size_t)nst * N * w->ns[s] * 8));
        }
        const int maxr = N > nsm ? N : nsm;
        w->nsm = nsm;
        CK(dalloc(A, &w->Ucur, 2 * (size_t)N * nsm * 8));
        CK(dalloc(A, &w->Utmp, (size_t)N * nsm * 8));
        CK(dalloc(A, &w->Ut2, 2 * (size_t)N * nsm * 8));
        CK(dalloc(A, &w->Ob, 2 * (size_t)nsm * nsm * 8));
        CK(dalloc(A, &w->Z, 2 * (size_t)nsm * N * 8));
        CK(dalloc(A, &w->Gnew, (size_t)N * ld * 8));
        CK(dalloc(A, (char**)&w->perm2, 2 * (size_t)maxr * sizeof(int)));
        CK(dalloc(A, (char**)&w->flag2, 2 * (size_t)maxr));
        CK(dalloc(A, (char**)&w->visited, (size_t)maxr * sizeof(int)));
        CK(dalloc(A, &w->acc2, 2 * 8));
        CK(cudaMemsetAsync(w->err, 0, sizeof(int), st));
        for (int q = 0; q < 2; ++q) {
            CK(cudaMemsetAsync(w->Wm[q], 0, 2 * (size_t)NW * NW * es, st));
            CK(cudaMemsetAsync(w->X[q], 0, 2 * (size_t)N * NW * es, st));
            CK(cudaMemsetAsync(w->Y[q], 0, 4 * (size_t)NW * N * es, st));
        }
        CK(cudaMemsetAsync(w->G, 0, 2 * (size_t)N * ld * es, st));
        CK(cudaMemsetAsync(w->Tbuf, 0, 2 * (size_t)N * ld * es, st));
        // fields
        if (fields) {
            CK(cudaMemcpyAsync(w->x, fields + foff, (size_t)M * N, cudaMemcpyHostToDevice, st));
            foff += (size_t)M * N;
        } else {
            count_launch();
            fields_kernel<<<(int)(((long)M * N + 255) / 256), 256, 0, st>>>(ctx->p.seed, (uint64_t)wi, (long)M * N, w->x);
            CK(cudaGetLastError());
        }
        count_launch();
        set_double_kernel<<<1, 1, 0, st>>>(w->sign, 1.0);
        CK(cudaGetLastError());
        // trial determinants -> stacks, G(0)  (Sec. II.B)
        double* ULc[2] = {w->Ucur, w->Ucur + (size_t)N * w->nsm};
        for (int s = 0; s < 2; ++s) {
            const int ns = w->ns[s];
            const double* Ph = P + poff;
            poff += (size_t)N * ns;
            // P into URs[s][0] (N x ns); its transpose starts the left stack, U_L(M) = P^T
            CK(cudaMemcpyAsync(w->URs[s], Ph, (size_t)N * ns * 8, cudaMemcpyHostToDevice, st));
            count_launch();
            transpose_kernel<<<256, 256, 0, st>>>(w->URs[s], N, ns, ULc[s]);
            CK(cudaGetLastError());
        }
        int grp[2][2], ng[2];
        const int ngr = spin_groups(w, grp, ng);
        for (int gi = 0; gi < ngr; ++gi) {
            double* R[2] = {w->URs[grp[gi][0]], ng[gi] > 1 ? w->URs[grp[gi][1]] : nullptr};
            double* Lc[2] = {ULc[grp[gi][0]], ng[gi] > 1 ? ULc[grp[gi][1]] : nullptr};
            CK(stab_rows(ctx, w, st, R, ng[gi], w->ns[grp[gi][0]], w->sign));
            CK(stab_cols(ctx, w, st, Lc, ng[gi], w->ns[grp[gi][0]], w->sign));
        }
        for (int s = 0; s < 2; ++s)
            CK(cudaMemcpyAsync(w->ULs[s] + (size_t)(M / S) * N * w->ns[s], ULc[s], (size_t)N * w->ns[s] * 8,
                               cudaMemcpyDeviceToDevice, st));
        // U_L(l - 1) = U_L(l) B_l, re-orthonormalised and stored at every recompute point
        for (int ell = M; ell >= 1; --ell) {
            if (ell % S == 0) CK(propagate(ctx, w, st, ULc, 1, ell, -1, S));  // slices ell .. ell - S + 1
            if ((ell - 1) % S == 0) {
                for (int gi = 0; gi < ngr; ++gi) {
                    double* Lc[2] = {ULc[grp[gi][0]], ng[gi] > 1 ? ULc[grp[gi][1]] : nullptr};
                    CK(stab_cols(ctx, w, st, Lc, ng[gi], w->ns[grp[gi][0]], w->sign));
                }
                for (int s = 0; s < 2; ++s)
                    CK(cudaMemcpyAsync(w->ULs[s] + (size_t)((ell - 1) / S) * N * w->ns[s], ULc[s],
                                       (size_t)N * w->ns[s] * 8, cudaMemcpyDeviceToDevice, st));
            }
        }
        // G(0) = 1 - U_R (U_L U_R)^{-1} U_L
        for (int gi = 0; gi < ngr; ++gi) {
            const double* R[2] = {w->URs[grp[gi][0]], ng[gi] > 1 ? w->URs[grp[gi][1]] : nullptr};
            const double* Lf[2] = {w->ULs[grp[gi][0]], ng[gi] > 1 ? w->ULs[grp[gi][1]] : nullptr};
            CK(form_Z(ctx, w, st, R, Lf, ng[gi], w->ns[grp[gi][0]], w->sign));
            for (int q = 0; q < ng[gi]; ++q) {
                const int s = grp[gi][q];
                CK(finish_G(w, st, w->URs[s], q, w->ns[s]));
                if (ctx->p.precision == AFQMC_PREC_FP64) CK(store_G<double>(w, st, s));
                else CK(store_G<float>(w, st, s));
            }
        }
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

template <typename T>
static int sweep_impl(afqmc_ctx* ctx, int wi, int ell, int dir, int mode, int k, int nb, const uint8_t* replay,
                      cudaStream_t st) {
    Walker* w = ctx->w[wi];
    const int N = w->N;
    const long ld = w->ld;
    T* G0 = (T*)w->G;
    T* G1 = G0 + (size_t)N * ld;
    T* Tb = (T*)w->Tbuf;
    int8_t* xl = w->x + (size_t)(ell - 1) * N;
    T* d = (T*)w->dvec;
    T* dinv = d + 2 * N;
    const T* E = (const T*)w->lat->Eb;
    const T* Einv = (const T*)w->lat->Einvb;
    const int NW = window_max<T>();
    const uint8_t* rep = nullptr;
    {
        PhaseScope ps(ctx, AFQMC_PHASE_PREP, st);
        CK(launch_uniforms(st, ctx->p.seed, (uint64_t)wi, w->visit, 2 * N, w->u));
        CK(cudaMemsetAsync(w->stats, 0, 8 * sizeof(int), st));
        CK(cudaMemsetAsync(w->maxr, 0, 8, st));
        if (replay) {
            CK(cudaMemcpyAsync(w->replay, replay + (size_t)wi * 2 * N, 2 * (size_t)N, cudaMemcpyHostToDevice, st));
            rep = w->replay;
        }
    }
    const bool use_tc = (sizeof(T) == 4) && ctx->p.gemm != AFQMC_GEMM_SIMT;
    const int split3 = ctx->p.gemm != AFQMC_GEMM_TF32;
    auto wrap = [&](int direction) -> cudaError_t {
        PhaseScope ps(ctx, AFQMC_PHASE_WRAP, st);
        cudaError_t e = launch_field_scales_T<T>(st, xl, N, ctx->c, d, dinv, N);
        if (e != cudaSuccess) return e;
        if (use_tc) {
            // E and Einv are symmetric, so both products are A * Bt^T with K-major operands:
            //   forward : S^T = (G Einv)^T ;  G = D (E S) D^{-1}
            //   backward: G <- D^{-1} G D ;  S^T = (G E)^T ;  G = Einv S
            const float* Ef = (const float*)E;
            const float* Eif = (const float*)Einv;
            float* Gf = (float*)G0;
            float* Tf = (float*)Tb;
            if (direction < 0) {
                e = launch_scale2<T>(st, G0, ld, N, (long)N * ld, dinv, d);
                if (e != cudaSuccess) return e;
            }
            TcGemmArgs t1;
            t1.M = N; t1.N = N; t1.K = N; t1.batch = 2;
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
            t2.M = N; t2.N = N; t2.K = N; t2.batch = 2;
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
        g1.M = N; g1.N = N; g1.K = N; g1.batch = 2;
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
    if (dir > 0) CK(wrap(+1));
    SiteParams sp;
    sp.N = N;
    sp.ld = ld;
    sp.c[0] = ctx->c[0];
    sp.c[1] = ctx->c[1];
    sp.lam = ctx->lam;
    sp.hs = ctx->p.hs;
    sp.seed = ctx->p.seed;
    sp.walker = (uint64_t)wi;
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
        PhaseScope ps(ctx, AFQMC_PHASE_LOCAL, st);
        CK(cudaMemsetAsync(w->bar, 0, sizeof(GridBar), st));
        CK(launch_local<T>(st, G0, G1, xl, w->u, rep, sp, so, (T*)w->colbuf, (T*)w->rowbuf, w->bar, w->err,
                           ctx->nsm));
    } else {
        int nw = (mode == AFQMC_MODE_DELAYED) ? k : (NW / nb) * nb;
        // Window w's decisions and the corrected block of window w + 1 run on st; window w's
        // panels and rank-m product run on the walker's flush stream sf and overlap the
        // decisions of window w + 1.  Before building window w + 1's block, st waits for the
        // product of window w - 1 (ev_prod), which is also what frees the window buffers of
        // parity (w + 1) & 1 for reuse.
        WindowBufs wb[2];
        for (int q = 0; q < 2; ++q) {
            wb[q].m = w->wm[q];
            wb[q].idx = w->widx[q];
            wb[q].dtot = w->wdtot[q];
            wb[q].Wm = w->Wm[q];
            wb[q].Wx = w->Wx[q];
            wb[q].X = w->X[q];
            wb[q].Y = w->Y[q];
        }
        PhaseScope ps(ctx, AFQMC_PHASE_CHAIN, st);
        int wi = 0;
        for (int s0 = 0; s0 < N; s0 += nw, ++wi) {
            const int n = (N - s0 < nw) ? N - s0 : nw;
            const int par = wi & 1;
            const T* blk = (wi > 0) ? (const T*)w->snap[par ^ 1] : nullptr;
            CK(launch_window_chain<T>(st, mode, G0, G1, xl, w->u, rep, sp, so, s0, n, nb, wb[par], blk, w->err));
            const int sn = s0 + n, nn = (sn < N) ? ((N - sn < nw) ? N - sn : nw) : 0;
            if (nn > 0) {  // the next window's block
                if (wi > 0) CK(cudaStreamWaitEvent(st, w->ev_prod[par ^ 1], 0));
                CK(launch_next_block<T>(st, G0, G1, sp, wb[par], sn, nn, (T*)w->snap[par]));
            }
            CK(cudaEventRecord(w->ev_chain[par], st));
            CK(cudaStreamWaitEvent(w->sf, w->ev_chain[par], 0));
            PhaseScope pf(ctx, AFQMC_PHASE_FLUSH, w->sf);
            CK(launch_flush_panels<T>(w->sf, G0, G1, sp, wb[par], n));
            {
                PhaseScope pg(ctx, AFQMC_PHASE_FLUSH_GEMM, w->sf);
                CK(launch_flush_gemm<T>(w->sf, G0, G1, sp, wb[par], n));
            }
            CK(cudaEventRecord(w->ev_prod[par], w->sf));
        }
        CK(cudaEventRecord(w->ev_done, w->sf));
        CK(cudaStreamWaitEvent(st, w->ev_done, 0));
    }
    if (dir < 0) CK(wrap(-1));
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
    for (auto* w : ctx->w) {
        if (w->need_recompute) return AFQMC_ERR_STATE;
        if (dir > 0 && w->pos != slice - 1) return AFQMC_ERR_STATE;
        if (dir < 0 && w->pos != slice) return AFQMC_ERR_STATE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    for (int wi = 0; wi < (int)ctx->w.size(); ++wi) {
        rc = f64 ? sweep_impl<double>(ctx, wi, slice, dir, mode, k, nb, replay, st)
                 : sweep_impl<float>(ctx, wi, slice, dir, mode, k, nb, replay, st);
        if (rc) return rc;
        Walker* w = ctx->w[wi];
        w->pos = (dir > 0) ? slice : slice - 1;
        w->last_dir = dir;
        w->visit++;
        if (w->pos % ctx->p.stab_every == 0) w->need_recompute = true;
    }
    if (stats) {
        CK(cudaStreamSynchronize(st));
        for (int wi = 0; wi < (int)ctx->w.size(); ++wi) {
            Walker* w = ctx->w[wi];
            int r = read_dev_err(ctx, w);
            if (r) return r;
            int h[8];
            CK(cudaMemcpy(h, w->stats, sizeof(h), cudaMemcpyDeviceToHost));
            stats[wi].proposals = h[0];
            stats[wi].accepts = h[1];
            stats[wi].flipped = h[2];
            stats[wi].flushes = h[3];
            CK(cudaMemcpy(&stats[wi].max_abs_ratio, w->maxr, 8, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(&stats[wi].sign, w->sign, 8, cudaMemcpyDeviceToHost));
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
    std::vector<double> drift(ctx->w.size(), 0.0);
    for (int wi = 0; wi < (int)ctx->w.size(); ++wi) {
        Walker* w = ctx->w[wi];
        const int N = w->N, j = w->pos / S;
        PhaseScope ps(ctx, AFQMC_PHASE_RECOMPUTE, st);
        CK(cudaMemsetAsync(w->acc2, 0, 16, st));
        // the factors of the current position: one side from the stacks, the other propagated
        // over the last S slices from the previous stack entry and re-orthonormalised
        double* UR[2];
        double* UL[2];
        double* Uc[2] = {w->Ucur, w->Ucur + (size_t)N * w->nsm};
        bool prop = false;
        for (int s = 0; s < 2; ++s) {
            const size_t blk = (size_t)N * w->ns[s];
            if (w->last_dir > 0) {
                UL[s] = w->ULs[s] + (size_t)j * blk;
                if (j == 0) {
                    UR[s] = w->URs[s];
                } else {
                    CK(cudaMemcpyAsync(Uc[s], w->URs[s] + (size_t)(j - 1) * blk, blk * 8, cudaMemcpyDeviceToDevice, st));
                    UR[s] = w->URs[s] + (size_t)j * blk;
                    prop = true;
                }
            } else {
                UR[s] = w->URs[s] + (size_t)j * blk;
                if (w->pos == ctx->p.M) {
                    UL[s] = w->ULs[s] + (size_t)j * blk;
                } else {
                    CK(cudaMemcpyAsync(Uc[s], w->ULs[s] + (size_t)(j + 1) * blk, blk * 8, cudaMemcpyDeviceToDevice, st));
                    UL[s] = w->ULs[s] + (size_t)j * blk;
                    prop = true;
                }
            }
        }
        int grp[2][2], ng[2];
        const int ngr = spin_groups(w, grp, ng);
        if (prop) {
            if (w->last_dir > 0) CK(propagate(ctx, w, st, Uc, 0, w->pos - S + 1, 1, S));
            else CK(propagate(ctx, w, st, Uc, 1, w->pos + S, -1, S));
            for (int gi = 0; gi < ngr; ++gi) {
                double* Cg[2] = {Uc[grp[gi][0]], ng[gi] > 1 ? Uc[grp[gi][1]] : nullptr};
                if (w->last_dir > 0) CK(stab_rows(ctx, w, st, Cg, ng[gi], w->ns[grp[gi][0]], nullptr));
                else CK(stab_cols(ctx, w, st, Cg, ng[gi], w->ns[grp[gi][0]], nullptr));
            }
            for (int s = 0; s < 2; ++s)
                CK(cudaMemcpyAsync(w->last_dir > 0 ? UR[s] : UL[s], Uc[s], (size_t)N * w->ns[s] * 8,
                                   cudaMemcpyDeviceToDevice, st));
        }
        for (int gi = 0; gi < ngr; ++gi) {
            const double* R[2] = {UR[grp[gi][0]], ng[gi] > 1 ? UR[grp[gi][1]] : nullptr};
            const double* Lf[2] = {UL[grp[gi][0]], ng[gi] > 1 ? UL[grp[gi][1]] : nullptr};
            CK(form_Z(ctx, w, st, R, Lf, ng[gi], w->ns[grp[gi][0]], nullptr));
            for (int q = 0; q < ng[gi]; ++q) {
                const int s = grp[gi][q];
                CK(finish_G(w, st, UR[s], q, w->ns[s]));
                if (f64) {
                    double* G = (double*)w->G + (size_t)s * N * w->ld;
                    CK(launch_drift<double>(st, G, (const double*)w->Gnew, w->ld, N, w->acc2));
                    CK(store_G<double>(w, st, s));
                } else {
                    float* G = (float*)w->G + (size_t)s * N * w->ld;
                    CK(launch_drift<float>(st, G, (const float*)w->Gnew, w->ld, N, w->acc2));
                    CK(store_G<float>(w, st, s));
                }
            }
        }
        w->need_recompute = false;
    }
    if (rel_drift) {
        CK(cudaStreamSynchronize(st));
        for (int wi = 0; wi < (int)ctx->w.size(); ++wi) {
            int r = read_dev_err(ctx, ctx->w[wi]);
            if (r) return r;
            double h[2];
            CK(cudaMemcpy(h, ctx->w[wi]->acc2, 16, cudaMemcpyDeviceToHost));
            rel_drift[wi] = h[1] > 0 ? sqrt(h[0] / h[1]) : 0.0;
        }
    }
    return AFQMC_OK;
}

int afqmc_measure_energy(afqmc_ctx* ctx, double* energy, double* sign, void* stream) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (ctx->w.empty() || !energy) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    for (auto* w : ctx->w) {
        CK(cudaMemsetAsync(w->acc2, 0, 16, st));
        if (ctx->p.precision == AFQMC_PREC_FP64) {
            const double* G = (const double*)w->G;
            CK(launch_energy<double>(st, G, G + (size_t)w->N * w->ld, w->ld, w->L, ctx->p.t, ctx->p.U, w->acc2));
        } else {
            const float* G = (const float*)w->G;
            CK(launch_energy<float>(st, G, G + (size_t)w->N * w->ld, w->ld, w->L, ctx->p.t, ctx->p.U, w->acc2));
        }
    }
    CK(cudaStreamSynchronize(st));
    for (int wi = 0; wi < (int)ctx->w.size(); ++wi) {
        Walker* w = ctx->w[wi];
        int r = read_dev_err(ctx, w);
        if (r) return r;
        CK(cudaMemcpy(&energy[wi], w->acc2, 8, cudaMemcpyDeviceToHost));
        if (sign) CK(cudaMemcpy(&sign[wi], w->sign, 8, cudaMemcpyDeviceToHost));
    }
    return AFQMC_OK;
}

int afqmc_get_G(afqmc_ctx* ctx, int walker, int spin, double* host_out) {
    if (!ctx || walker < 0 || walker >= (int)ctx->w.size() || spin < 0 || spin > 1 || !host_out) return AFQMC_ERR_ARG;
    Walker* w = ctx->w[walker];
    CK(cudaStreamSynchronize(ctx->last));
    const size_t es = esize(ctx);
    std::vector<char> buf((size_t)w->N * w->ld * es);
    CK(cudaMemcpy(buf.data(), (char*)w->G + (size_t)spin * w->N * w->ld * es, buf.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < w->N; ++i)
        for (int j = 0; j < w->N; ++j) {
            size_t o = (size_t)i * w->ld + j;
            host_out[(size_t)i * w->N + j] = (es == 8) ? ((double*)buf.data())[o] : (double)((float*)buf.data())[o];
        }
    return read_dev_err(ctx, w);
}

int afqmc_set_G(afqmc_ctx* ctx, int walker, int spin, const double* host_in) {
    if (!ctx || walker < 0 || walker >= (int)ctx->w.size() || spin < 0 || spin > 1 || !host_in) return AFQMC_ERR_ARG;
    Walker* w = ctx->w[walker];
    CK(cudaStreamSynchronize(ctx->last));
    const size_t es = esize(ctx);
    std::vector<char> buf((size_t)w->N * w->ld * es, 0);
    for (int i = 0; i < w->N; ++i)
        for (int j = 0; j < w->N; ++j) {
            size_t o = (size_t)i * w->ld + j;
            double v = host_in[(size_t)i * w->N + j];
            if (es == 8) ((double*)buf.data())[o] = v;
            else ((float*)buf.data())[o] = (float)v;
        }
    CK(cudaMemcpy((char*)w->G + (size_t)spin * w->N * w->ld * es, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    return AFQMC_OK;
}

int afqmc_get_fields(afqmc_ctx* ctx, int walker, int8_t* host_out) {
    if (!ctx || walker < 0 || walker >= (int)ctx->w.size() || !host_out) return AFQMC_ERR_ARG;
    Walker* w = ctx->w[walker];
    CK(cudaStreamSynchronize(ctx->last));
    CK(cudaMemcpy(host_out, w->x, (size_t)ctx->p.M * w->N, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

int afqmc_get_decisions(afqmc_ctx* ctx, int walker, uint8_t* host_out) {
    if (!ctx || walker < 0 || walker >= (int)ctx->w.size() || !host_out) return AFQMC_ERR_ARG;
    Walker* w = ctx->w[walker];
    CK(cudaStreamSynchronize(ctx->last));
    CK(cudaMemcpy(host_out, w->dec, 2 * (size_t)w->N, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

int afqmc_get_ratios(afqmc_ctx* ctx, int walker, double* host_out) {
    if (!ctx || walker < 0 || walker >= (int)ctx->w.size() || !host_out) return AFQMC_ERR_ARG;
    Walker* w = ctx->w[walker];
    CK(cudaStreamSynchronize(ctx->last));
    CK(cudaMemcpy(host_out, w->ratio, 2 * (size_t)w->N * 8, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

int afqmc_get_info(afqmc_ctx* ctx, int walker, int* N, int* n_up, int* n_dn, int* slice, int* dir) {
    if (!ctx || walker < 0 || walker >= (int)ctx->w.size()) return AFQMC_ERR_ARG;
    Walker* w = ctx->w[walker];
    if (N) *N = w->N;
    if (n_up) *n_up = w->ns[0];
    if (n_dn) *n_dn = w->ns[1];
    if (slice) *slice = w->pos;
    if (dir) *dir = w->last_dir;
    return AFQMC_OK;
}

int afqmc_set_profiling(afqmc_ctx* ctx, int on) {
    if (!ctx) return AFQMC_ERR_ARG;
    if (ctx->last) cudaStreamSynchronize(ctx->last);
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
    CK(cudaStreamSynchronize(ctx->last));
    for (auto* w : ctx->w)
        if (w->sf) CK(cudaStreamSynchronize(w->sf));
    for (auto& pe : ctx->prof.pending) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, pe.a, pe.b));
        ctx->prof.ms[pe.phase] += t;
        ctx->prof.intervals[pe.phase] += 1;
        ctx->prof.pool.push_back(pe.a);
        ctx->prof.pool.push_back(pe.b);
    }
    ctx->prof.pending.clear();
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
