// Host build of the separable-wrap tile code (paper_2506_09611_gb300/csrc/sepwrap.cuh) for the CPU
// tests: every tile of every matrix runs serially as one "thread" with no-op barriers (each phase
// of the tile reads one buffer and writes another, so the serial order gives the block's result).
#include <vector>

#include "../paper_2506_09611_gb300/csrc/sepwrap.cuh"

namespace {
struct NoSync {
    void operator()() const {}
};

template <typename T>
void run(const afq::SepArgs& a) {
    std::vector<unsigned char> smem(afq::sep_smem_bytes<T>(a.L, a.N, a.w));
    const int ntiles = ((a.C > 0 ? a.C : a.N) + a.w - 1) / a.w;
    for (int z = 0; z < a.batch; ++z)
        for (int t = 0; t < ntiles; ++t) afq::sep_tile<T>(a, t, z, 0, 1, smem.data(), NoSync());
}
}  // namespace

// One pass (side 0 or 1) with tile width w on N x C (side 0) or C x N (side 1) matrices (C = 0:
// square); the scale pointers are nullable.
extern "C" void sep_host_pass(int fp64, int side, int L, int C, int w, int batch, void* G, long ld, long sG,
                              const double* A, const void* rs_in, const void* cs_in, const void* rs_out,
                              const void* cs_out, long sv) {
    afq::SepArgs a;
    a.G = G; a.ld = ld; a.sG = sG; a.L = L; a.N = L * L; a.C = C; a.batch = batch; a.A = A; a.side = side; a.w = w;
    a.rs_in = rs_in; a.cs_in = cs_in; a.rs_out = rs_out; a.cs_out = cs_out; a.sv = sv;
    if (fp64) run<double>(a); else run<float>(a);
}

// Vector accesses so far that would be misaligned on the device (must stay 0).
extern "C" int sep_host_misaligned() { return afq::sep_misaligned_count(); }

// The wrap as the library issues it (sep_wrap_passes), tile width w.
extern "C" void sep_host_wrap(int fp64, int direction, int L, int w, int batch, void* G, long ld, long sG,
                              const double* Ex, const double* Exi, const void* d, const void* dinv, long sv) {
    afq::SepArgs a1, a2;
    afq::sep_wrap_passes(direction, G, ld, sG, L, batch, Ex, Exi, d, dinv, sv, &a1, &a2);
    a1.w = a2.w = w;
    if (fp64) { run<double>(a1); run<double>(a2); } else { run<float>(a1); run<float>(a2); }
}
