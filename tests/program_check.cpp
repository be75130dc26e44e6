// Host build of a generated diagram program in double precision, for the CPU
// tests of the code generator: the colour-summed |M|^2 of one helicity
// (helicity_msq) and of a helicity pair (helicity_pair_msq) at given momenta.
// The generated source, cut before its kernel, is included as
// "mf_program_gen.h" (the test writes it next to this build).
//
// stdin: n_masses masses..., n_couplings (re im)..., then lines
//   msq  h_0 .. h_{n-1}  p_0^0 .. p_{n-1}^3     ->  |M_h|^2
//   pair h_0 .. h_{n-1}  p_0^0 .. p_{n-1}^3     ->  |M_a|^2 |M_b|^2
// (a: the row with the pair leg at -1, b: at +1)
#include <cstdint>

#define __device__
#define __noinline__
#define MF_PROG_SYNC()
// the device headers' 64-bit high product (Philox), for the host
static inline uint64_t __umul64hi(uint64_t a, uint64_t b) {
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
}
#include "mf_program_gen.h"

#include <cstdio>
#include <cstring>
#include <vector>

int main() {
    int nm = 0, nc = 0;
    if (std::scanf("%d", &nm) != 1 || nm < 0 || nm > 8) return 1;
    std::vector<double> mass(8, 0.0);
    for (int i = 0; i < nm; ++i)
        if (std::scanf("%lf", &mass[i]) != 1) return 1;
    if (std::scanf("%d", &nc) != 1 || nc < 0 || nc > 8) return 1;
    std::vector<mf::cx<double>> cpl(8, mf::cx<double>{0.0, 0.0});
    for (int i = 0; i < nc; ++i)
        if (std::scanf("%lf %lf", &cpl[i].re, &cpl[i].im) != 2) return 1;
    constexpr int N = proc::NLEG, ND = proc::NDEN > 0 ? proc::NDEN : 1;
    char cmd[16];
    while (std::scanf("%15s", cmd) == 1) {
        int8_t hel[N];
        for (int l = 0; l < N; ++l) {
            int h = 0;
            if (std::scanf("%d", &h) != 1) return 1;
            hel[l] = (int8_t)h;
        }
        double p[N][4], ms[4 * N], den[ND], idn[ND];
        for (int l = 0; l < N; ++l)
            for (int q = 0; q < 4; ++q) {
                if (std::scanf("%lf", &p[l][q]) != 1) return 1;
                ms[4 * l + q] = p[l][q];
            }
        proc::denominators<double>(p, mass.data(), den);
        for (int k = 0; k < ND; ++k) idn[k] = 1.0 / den[k];
        if (std::strcmp(cmd, "msq") == 0) {
            std::printf("%.17g\n", proc::helicity_msq<double>(ms, idn, hel, cpl.data(), mass.data()));
        } else {
            double va = 0.0, vb = 0.0;
            proc::helicity_pair_msq<double>(ms, idn, hel, cpl.data(), mass.data(), va, vb);
            std::printf("%.17g %.17g\n", va, vb);
        }
    }
    return 0;
}
