// Host build of the separable-wrap code (paper_2506_09611_gb300/csrc/sepwrap.cuh) for the CPU
// tests: every tile of every matrix runs serially as one "thread" with no-op barriers (each phase
// of the tile reads one buffer and writes another, so the serial order gives the block's result),
// and the line passes run line by line (each line is read into registers before it is written).
#include <vector>

#include "../paper_2506_09611_gb300/csrc/sepwrap.cuh"

namespace {
struct NoSync {
    void operator()() const {}
};

template <typename T, int LM>
void run_line(const afq::SepLineArgs& p, const double* A) {
    alignas(16) T As[LM * LM];
    afq::sep_line_load_A<T>(A, p.L, LM, As, 0, 1);
    const long total = afq::sep_line_count(p) * p.batch;
    for (long line = 0; line < total; ++line) afq::sep_line<T, LM>(p, line, As);
}

template <typename T, int L>
void run_circ(const afq::SepLineArgs& p, const double* A) {
    T c[L];
    for (int d = 0; d < L; ++d) c[d] = (T)A[d];  // the kernel's registers
    const long total = afq::sep_line_count(p) * p.batch;
    for (long line = 0; line < total; ++line) afq::sep_line_circ<T, L>(p, line, c);
}

template <typename T>
void run_line_lm(const afq::SepLineArgs& p, const double* A) {
    if (p.circ && afq::sep_circ_side<T>(p.L)) {
        switch (p.L) {
            case 4: run_circ<T, 4>(p, A); break;
            case 6: run_circ<T, 6>(p, A); break;
            case 8: run_circ<T, 8>(p, A); break;
            case 12: run_circ<T, 12>(p, A); break;
            case 16: run_circ<T, 16>(p, A); break;
            case 20: run_circ<T, 20>(p, A); break;
            case 24: run_circ<T, 24>(p, A); break;
            case 32: run_circ<T, 32>(p, A); break;
            case 40: run_circ<T, 40>(p, A); break;
            default: break;
        }
        return;
    }
    switch (afq::sep_line_lm(p.L)) {
        case 8: run_line<T, 8>(p, A); break;
        case 12: run_line<T, 12>(p, A); break;
        case 16: run_line<T, 16>(p, A); break;
        case 20: run_line<T, 20>(p, A); break;
        case 24: run_line<T, 24>(p, A); break;
        case 32: run_line<T, 32>(p, A); break;
        case 40: run_line<T, 40>(p, A); break;
        case 48: run_line<T, 48>(p, A); break;
        case 64: run_line<T, 64>(p, A); break;
        default: break;
    }
}

// As the device launcher dispatches: w == 0 takes the two line passes, w > 0 tiles of w columns.
template <typename T>
void run(const afq::SepArgs& a) {
    if (a.w == 0) {
        afq::SepLineArgs p1, p2;
        afq::sep_line_passes(a, &p1, &p2);
        run_line_lm<T>(p1, a.A);
        run_line_lm<T>(p2, a.A);
        return;
    }
    std::vector<unsigned char> smem(afq::sep_smem_bytes<T>(a.L, a.N, a.w));
    const int ntiles = ((a.C > 0 ? a.C : a.N) + a.w - 1) / a.w;
    for (int z = 0; z < a.batch; ++z)
        for (int t = 0; t < ntiles; ++t) afq::sep_tile<T>(a, t, z, 0, 1, smem.data(), NoSync());
}
}  // namespace

// One pass (side 0 or 1) with tile width w (0: the two line passes) on N x C (side 0) or C x N
// (side 1) matrices (C = 0: square); the scale pointers are nullable; circ: A is circulant (the
// line passes may use its first row).
extern "C" void sep_host_pass(int fp64, int side, int L, int C, int w, int batch, void* G, long ld, long sG,
                              const double* A, const void* rs_in, const void* cs_in, const void* rs_out,
                              const void* cs_out, long sv, int circ) {
    afq::SepArgs a;
    a.circ = circ;
    a.G = G; a.ld = ld; a.sG = sG; a.L = L; a.N = L * L; a.C = C; a.batch = batch; a.A = A; a.side = side; a.w = w;
    a.rs_in = rs_in; a.cs_in = cs_in; a.rs_out = rs_out; a.cs_out = cs_out; a.sv = sv;
    if (fp64) run<double>(a); else run<float>(a);
}

// Vector accesses so far that would be misaligned on the device (must stay 0).
extern "C" int sep_host_misaligned() { return afq::sep_misaligned_count(); }

// The wrap as the library issues it (sep_wrap_passes), tile width w (0: line passes).
extern "C" void sep_host_wrap(int fp64, int direction, int L, int w, int batch, void* G, long ld, long sG,
                              const double* Ex, const double* Exi, const void* d, const void* dinv, long sv) {
    afq::SepArgs a1, a2;
    afq::sep_wrap_passes(direction, G, ld, sG, L, batch, Ex, Exi, d, dinv, sv, &a1, &a2);
    a1.w = a2.w = w;
    if (fp64) { run<double>(a1); run<double>(a2); } else { run<float>(a1); run<float>(a2); }
}
