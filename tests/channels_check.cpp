// Host build of the device channel header (csrc/device/mf_channels.cuh) for
// CPU tests: reads commands from stdin, prints results with 17 significant
// digits.
//   table L t_0 .. t_{L-1}                       -> (load a channel table)
//   gen n ch rs s0 t0 m_t fm_0..fm_{n-1} u_0..u_{3n-5}
//                                                 -> ok 1/g share p_00 .. p_{n-1,3}
//   gend (same arguments)                         -> ok, then 1/g, share, p_00 .. p_{n-1,3},
//                                                    each as a value and its derivatives with
//                                                    respect to u_0 .. u_{3n-5} and m_t
//                                                    (the top legs' masses are m_t)
#include <cstdint>
#include <cstdio>
#include <iostream>
#include <sstream>
#include <string>
#include <vector>

#include "mf_channels.cuh"

static std::vector<int32_t> g_table;

template <int N>
static void gen(std::istringstream &in) {
    int ch;
    double rs, s0, t0, mt, fm[N], u[3 * N - 4], p[N][4];
    in >> ch >> rs >> s0 >> t0 >> mt;
    for (int i = 0; i < N; ++i) in >> fm[i];
    for (int i = 0; i < 3 * N - 4; ++i) in >> u[i];
    const double masses[1] = {mt};
    double inv_g = 0.0;
    const bool ok = mf::channel_generate<N>(g_table.data(), ch, u, rs, fm, masses, s0, t0, p, inv_g);
    const double share = mf::channel_share<N>(g_table.data(), ch, rs, p, masses, s0, t0);
    std::printf("%d %.17g %.17g", ok ? 1 : 0, inv_g, share);
    for (int i = 0; i < N; ++i)
        for (int q = 0; q < 4; ++q) std::printf(" %.17g", p[i][q]);
    std::printf("\n");
}

template <int N>
static void gend(std::istringstream &in) {
    constexpr int K = 3 * N - 3;              // the 3N-4 unit numbers and m_t
    using D = mf::Dual<K>;
    int ch;
    double rs, s0, t0, mt, fmv[N], uv[3 * N - 4];
    in >> ch >> rs >> s0 >> t0 >> mt;
    for (int i = 0; i < N; ++i) in >> fmv[i];
    for (int i = 0; i < 3 * N - 4; ++i) in >> uv[i];
    D u[3 * N - 4], fm[N], p[N][4];
    for (int i = 0; i < 3 * N - 4; ++i) u[i] = D::seed(uv[i], i);
    const D m = D::seed(mt, K - 1);
    for (int i = 0; i < N; ++i) fm[i] = fmv[i] > 0.0 ? m : D(0.0);
    const D masses[1] = {m};
    D inv_g(0.0);
    const bool ok = mf::channel_generate<N, D>(g_table.data(), ch, u, D(rs), fm, masses, s0, t0, p, inv_g);
    const D share = mf::channel_share<N, D>(g_table.data(), ch, D(rs), p, masses, s0, t0);
    auto put = [](const D &x) {
        std::printf(" %.17g", x.v);
        for (int k = 0; k < K; ++k) std::printf(" %.17g", x.d[k]);
    };
    std::printf("%d", ok ? 1 : 0);
    put(inv_g);
    put(share);
    for (int i = 0; i < N; ++i)
        for (int q = 0; q < 4; ++q) put(p[i][q]);
    std::printf("\n");
}

int main() {
    std::string line;
    while (std::getline(std::cin, line)) {
        std::istringstream in(line);
        std::string cmd;
        in >> cmd;
        if (cmd == "table") {
            int n;
            in >> n;
            g_table.assign(n, 0);
            for (int i = 0; i < n; ++i) in >> g_table[i];
        } else if (cmd == "gend") {
            int n;
            in >> n;
            switch (n) {
                case 2: gend<2>(in); break;
                case 3: gend<3>(in); break;
                case 4: gend<4>(in); break;
                default: std::printf("bad n\n");
            }
        } else if (cmd == "gen") {
            int n;
            in >> n;
            switch (n) {
                case 2: gen<2>(in); break;
                case 3: gen<3>(in); break;
                case 4: gen<4>(in); break;
                case 5: gen<5>(in); break;
                case 6: gen<6>(in); break;
                default: std::printf("bad n\n");
            }
        }
        std::fflush(stdout);
    }
    return 0;
}
