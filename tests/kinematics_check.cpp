// Host build of the device kinematics header (csrc/device/mf_kinematics.cuh)
// for CPU tests: reads commands from stdin and prints results with 17
// significant digits.
//   ratio m r                 -> x d          (mass ratio and its complement)
//   philox c0 c1 c2 c3 k0 k1  -> four 64-bit outputs
//   diet n rs u_1 .. u_{3n-4} -> n x 4 momentum components
#include <cstdint>
#include <cstdio>
#include <iostream>
#include <sstream>
#include <string>

// the one device intrinsic the header uses, for a host build
static inline uint64_t __umul64hi(uint64_t a, uint64_t b) {
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
}
#include "mf_kinematics.cuh"

template <int N>
static void diet(std::istringstream &in) {
    double rs, u[3 * N - 4], p[N][4];
    in >> rs;
    for (int i = 0; i < 3 * N - 4; ++i) in >> u[i];
    mf::massless_diet<N, double>(u, rs, p);
    for (int i = 0; i < N; ++i)
        for (int q = 0; q < 4; ++q) std::printf("%.17g ", p[i][q]);
    std::printf("\n");
}

int main() {
    std::string line;
    while (std::getline(std::cin, line)) {
        std::istringstream in(line);
        std::string cmd;
        in >> cmd;
        if (cmd == "ratio") {
            int m;
            double r, d;
            in >> m >> r;
            double x = mf::mass_ratio(m, r, d);
            std::printf("%.17g %.17g\n", x, d);
        } else if (cmd == "philox") {
            uint64_t c[4], k0, k1;
            in >> c[0] >> c[1] >> c[2] >> c[3] >> k0 >> k1;
            mf::philox4x64_10(c, k0, k1);
            std::printf("%llu %llu %llu %llu\n", (unsigned long long)c[0], (unsigned long long)c[1],
                        (unsigned long long)c[2], (unsigned long long)c[3]);
        } else if (cmd == "diet") {
            int n;
            in >> n;
            if (n == 2) diet<2>(in);
            else if (n == 3) diet<3>(in);
            else if (n == 4) diet<4>(in);
            else if (n == 5) diet<5>(in);
            else if (n == 6) diet<6>(in);
            else std::printf("bad n\n");
        } else {
            std::printf("bad command\n");
        }
    }
    return 0;
}
