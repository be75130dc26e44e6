// Code generation: the diagram program of an mf_process becomes straight-line
// CUDA (one function per helicity evaluation), so that every wavefunction lives
// in registers and every routine is inlined.  This replaces the paper's
// exporter to TensorFlow (Sec. 2.2) with specialisation at run time.
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <functional>
#include <algorithm>
#include <map>
#include <sstream>

#include "mf_internal.h"

namespace mfi {
bool large_program(const mf_process &p);
namespace {

std::string fmt_double(double v) {
    char buf[64];
    std::snprintf(buf, sizeof buf, "%.17g", v);
    std::string s(buf);
    if (s.find_first_of(".eEn") == std::string::npos) s += ".0";
    return s;
}

// algorithmic FLOPs of each routine as written in mf_helas.cuh (fma = 2)
double routine_flops(int r) {
    switch (r) {
        case MF_R_IXX: case MF_R_OXX: return 40;
        case MF_R_VXX: return 30;
        case MF_R_FFV_AMP: return 100;
        case MF_R_FFV_FIN: return 160;
        case MF_R_FFV_FOUT: return 164;
        case MF_R_FFV_VEC: return 150;
        case MF_R_VVV_AMP: return 172;
        case MF_R_VVV_VEC: return 180;
        case MF_R_VVVV1_AMP: case MF_R_VVVV2_AMP: case MF_R_VVVV3_AMP: return 140;
        case MF_R_VVVV1_VEC: case MF_R_VVVV2_VEC: case MF_R_VVVV3_VEC: return 155;
        default: return 0;
    }
}

// FLOPs of one op's routine as emitted: a coupling that is real or
// imaginary (pmul) turns each product with the coupling factor into a
// real-times-complex one, 4 FLOPs fewer (four per current, one per
// amplitude)
double op_flops(const mf_process &p, const mf_op &op) {
    double f = routine_flops(op.routine);
    const int c = op.coupling;
    if (op.kind == MF_OP_EXT || c < 0 || 2 * c + 1 >= (int)p.couplings.size()) return f;
    const double re = p.couplings[2 * c], im = p.couplings[2 * c + 1];
    if (re != 0.0 && im != 0.0) return f;
    return f - (op.kind == MF_OP_CUR ? 16.0 : 4.0);
}

// an amplitude's colour coefficients as emitted: a complex add for +-1 and
// +-i, a complex multiply-add otherwise
double term_flops(const mf_process &p, const mf_op &op) {
    double f = 0.0;
    for (int t = 0; t < op.n_terms; ++t) {
        const mf_colour_term &ct = p.terms[op.first_term + t];
        const bool unit = (ct.im == 0.0 && (ct.re == 1.0 || ct.re == -1.0)) ||
                          (ct.re == 0.0 && (ct.im == 1.0 || ct.im == -1.0));
        f += unit ? 2.0 : 8.0;
    }
    return f;
}

// the colour sum as emitted: per flow a real-times-complex product, per
// non-zero entry above the diagonal a real-times-complex multiply-add, per
// flow the real part of conj(J_k) z (leading colour: c_kk |J_k|^2 per flow)
double colour_sum_flops(const mf_process &p) {
    const int nj = p.n_jamp;
    if (p.leading_colour) return 5.0 * nj;        // the diagonal only: c_kk |J_k|^2
    double f = 6.0 * nj;
    for (int k = 0; k < nj; ++k)
        for (int l = k + 1; l < nj; ++l)
            if (p.colour_num[k * nj + l] != 0) f += 4.0;
    return f;
}

// FFV amplitudes that share the row and column spinors and the coupling
// and whose colour coefficients agree up to a factor +-1 or +-i form one
// unit: the amplitude is linear in its vector current, so the unit's members
// contribute c_k(first) * FFV(row, col, sum_a phi_a V_a), phi_a the member's
// factor (0: 1, 1: i, 2: -1, 3: -i).  Every other amplitude is a unit alone.
struct AmpUnit {
    std::vector<int> ops;
    std::vector<int> phase;
    int ph0 = 0;                  // phase of the first member's lowest-flow coefficient
};

std::vector<AmpUnit> amplitude_units(const mf_process &p) {
    std::vector<AmpUnit> units;
    // used for every program unless the process options say otherwise (0:
    // every amplitude alone, 1: units); measured on GB300: gg -> tt~gg 1.13x,
    // gg -> tt~g 1.03x (mixed) and 1.08x (FP64)
    bool group = true;
    if (p.opt.amplitude_units >= 0) group = p.opt.amplitude_units != 0;
    std::map<std::vector<double>, int> unit_of;
    auto unit_phase = [](double re, double im) {
        if (im == 0.0 && re == 1.0) return 0;
        if (re == 0.0 && im == 1.0) return 1;
        if (im == 0.0 && re == -1.0) return 2;
        if (re == 0.0 && im == -1.0) return 3;
        return -1;
    };
    for (size_t k = 0; k < p.ops.size(); ++k) {
        const mf_op &op = p.ops[k];
        if (op.kind != MF_OP_AMP) continue;
        int ph = -1;
        std::vector<double> key;
        if (group && op.routine == MF_R_FFV_AMP && op.n_terms > 0) {
            std::vector<std::pair<int, std::pair<double, double>>> t;
            for (int q = 0; q < op.n_terms; ++q) {
                const mf_colour_term &ct = p.terms[op.first_term + q];
                t.push_back({ct.jamp, {ct.re, ct.im}});
            }
            std::sort(t.begin(), t.end());
            ph = unit_phase(t[0].second.first, t[0].second.second);
            if (ph >= 0) {
                // divide by the first coefficient (exact for a unit phase)
                const double cr = t[0].second.first, ci = -t[0].second.second;
                key = {(double)op.in[0], (double)op.in[1], (double)op.coupling};
                for (auto &e : t) {
                    key.push_back(e.first);
                    key.push_back(e.second.first * cr - e.second.second * ci);
                    key.push_back(e.second.first * ci + e.second.second * cr);
                }
            }
        }
        if (ph >= 0) {
            auto it = unit_of.find(key);
            if (it != unit_of.end()) {
                AmpUnit &u = units[it->second];
                u.ops.push_back((int)k);
                u.phase.push_back((ph - u.ph0 + 4) % 4);
                continue;
            }
            unit_of[key] = (int)units.size();
        }
        units.push_back(AmpUnit{{(int)k}, {0}, ph >= 0 ? ph : 0});
    }
    return units;
}

// Peak number of internal wavefunctions live at once when the units are
// emitted in `order` (each unit's wavefunctions just before it, a
// wavefunction live from its definition to its last use), and the sum of the
// live counts over the emission steps (a tie-breaker).
std::pair<int, long> live_profile(const mf_process &p, const std::vector<AmpUnit> &units,
                                  const std::vector<int> &order) {
    const size_t n = p.ops.size();
    std::vector<int> def(n, -1), last(n, -1);
    int t = 0;
    std::function<void(int)> emit = [&](int k) {
        if (def[k] >= 0) return;
        for (int q = 0; q < 4; ++q)
            if (p.ops[k].in[q] >= 0) emit(p.ops[k].in[q]);
        for (int q = 0; q < 4; ++q)
            if (p.ops[k].in[q] >= 0) last[p.ops[k].in[q]] = t;
        def[k] = t++;
    };
    for (int u : order) {
        for (int a : units[u].ops)
            for (int q = 0; q < 4; ++q)
                if (p.ops[a].in[q] >= 0) emit(p.ops[a].in[q]);
        for (int a : units[u].ops)
            for (int q = 0; q < 4; ++q)
                if (p.ops[a].in[q] >= 0) last[p.ops[a].in[q]] = t;
        ++t;
    }
    std::vector<int> ev(t + 2, 0);
    for (size_t k = 0; k < n; ++k)
        if (def[k] >= 0 && p.ops[k].kind == MF_OP_CUR) {
            ev[def[k]]++;
            ev[(last[k] >= 0 ? last[k] : def[k]) + 1]--;
        }
    int cur = 0, peak = 0;
    long sum = 0;
    for (int v : ev) {
        cur += v;
        peak = std::max(peak, cur);
        sum += cur;
    }
    return {peak, sum};
}

// Local search on the unit order: move one unit to another position and
// keep the move when the peak (then the sum) of live wavefunctions does not
// grow.  A fixed-seed generator keeps the result, and so the generated
// source and its cached binary, reproducible.
void improve_order(const mf_process &p, const std::vector<AmpUnit> &units, std::vector<int> &order, int iters) {
    if (order.size() < 3) return;
    auto best = live_profile(p, units, order);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    auto next = [&](uint64_t m) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        return (st >> 33) % m;
    };
    for (int it = 0; it < iters; ++it) {
        std::vector<int> o = order;
        const size_t i = next(o.size());
        const int u = o[i];
        o.erase(o.begin() + i);
        o.insert(o.begin() + next(o.size() + 1), u);
        auto s = live_profile(p, units, o);
        if (s <= best) {
            best = s;
            order.swap(o);
        }
    }
}

}  // namespace

// FLOPs of the wavefunctions whose momentum does not flow through `leg`
// (the part of the program two helicities differing only at `leg` share).
double shared_flops(const mf_process &p, int leg) {
    std::vector<uint32_t> m(p.ops.size(), 0);
    double f = 0.0;
    for (size_t k = 0; k < p.ops.size(); ++k) {
        const mf_op &op = p.ops[k];
        if (op.kind == MF_OP_AMP) continue;
        if (op.kind == MF_OP_EXT) m[k] = 1u << op.leg;
        for (int q = 0; q < 4; ++q)
            if (op.in[q] >= 0) m[k] |= m[op.in[q]];
        if (!(m[k] >> leg & 1)) f += routine_flops(op.routine);
    }
    return f;
}

// A program long enough to be bound by instruction fetch (the diagram
// program of one helicity above 2e4 FLOPs; gg -> tt~gg has 4.7e4).
bool large_program(const mf_process &p) {
    double f = 0.0;
    for (const mf_op &op : p.ops) f += routine_flops(op.routine);
    return f >= 2e4;
}

// The leg whose helicity the fewest wavefunctions depend on (the most FLOPs
// shared by a pair of helicities differing only there; lowest index on
// ties), or -1 if no current is independent of every leg.
int pair_leg(const mf_process &p) {
    // no pair program when the option turns pairs off, and by default for
    // programs above 1.5e5 FLOPs per helicity (gg -> tt~ggg: 3.7e5), whose
    // single-helicity program alone takes minutes to compile
    if (p.opt.helicity_pairs == 0) return -1;
    if (p.opt.helicity_pairs < 0) {
        double f = 0.0;
        for (const mf_op &op : p.ops) f += routine_flops(op.routine);
        if (f >= 1.5e5) return -1;
    }
    int best = -1;
    double bf = 0.0;
    for (int l = 0; l < p.n_legs; ++l) {
        double f = shared_flops(p, l);
        // the other legs' external wavefunctions alone are not worth a pair
        double ext = 0.0;
        for (const mf_op &op : p.ops)
            if (op.kind == MF_OP_EXT && op.leg != l) ext += routine_flops(op.routine);
        if (f > ext && f > bf) { best = l; bf = f; }
    }
    return best;
}

// Includes, the process constants and the double-precision propagator
// denominators (shared by the integrand and the gradient sources).
void emit_header(std::ostringstream &o, const mf_process &p, GenInfo &info, std::vector<uint32_t> &mask,
                 const char *R, const char *ns = "proc") {
    const int n = p.n_legs;
    // --- wavefunction momenta as signed leg masks, denominator slots
    mask.assign(p.ops.size(), 0);
    info = GenInfo{};
    info.op_den.assign(p.ops.size(), -1);
    std::map<std::pair<uint32_t, int>, int> slot_of;
    for (size_t k = 0; k < p.ops.size(); ++k) {
        const mf_op &op = p.ops[k];
        if (op.kind == MF_OP_EXT) {
            mask[k] = 1u << op.leg;
        } else if (op.kind == MF_OP_CUR) {
            uint32_t m = 0;
            for (int q = 0; q < 4; ++q)
                if (op.in[q] >= 0) m |= mask[op.in[q]];
            mask[k] = m;
            auto key = std::make_pair(m, (int)op.mass_id);
            auto it = slot_of.find(key);
            if (it == slot_of.end()) {
                int s = (int)info.dens.size();
                info.dens.push_back(DenSlot{m, op.mass_id});
                slot_of[key] = s;
                info.op_den[k] = s;
            } else {
                info.op_den[k] = it->second;
            }
        }
    }
    info.n_den = (int)info.dens.size();

    o << "// generated: diagram program of one process, precision " << R << "\n";
    o << "#include \"mf_common.cuh\"\n#include \"mf_kinematics.cuh\"\n#include \"mf_helas.cuh\"\n";
    o << "#ifndef MF_PROG_SYNC\n#define MF_PROG_SYNC() __syncthreads()\n#endif\n";
    o << "namespace " << ns << " {\n";
    o << "constexpr bool LEADING_COLOUR = " << (p.leading_colour ? "true" : "false") << ";\n";
    o << "constexpr int NLEG = " << n << ", NOUT = " << p.n_out << ", NDIM = " << p.ndim
      << ", NJAMP = " << p.n_jamp << ", NDEN = " << info.n_den << ", HADRONIC = " << p.hadronic << ";\n";
    o << "__device__ constexpr int LEG_MASS_ID[NLEG] = {";
    for (int i = 0; i < n; ++i) o << (i ? ", " : "") << p.leg_mass_id[i];
    o << "};\n";
    std::vector<int> cuts;
    for (int i = 0; i < n; ++i)
        if (p.leg_cut[i] && !p.leg_incoming[i]) cuts.push_back(i);
    o << "constexpr int NCUT = " << cuts.size() << ";\n";
    o << "__device__ constexpr int CUT_LEGS[" << (cuts.empty() ? 1 : cuts.size()) << "] = {";
    if (cuts.empty()) o << "0";
    for (size_t i = 0; i < cuts.size(); ++i) o << (i ? ", " : "") << cuts[i];
    o << "};\n";

    // --- propagator denominators from double-precision invariants
    o << "template <typename T>\nMF_DEV void denominators(const T (*p)[4], const T *masses, T *den) {\n";
    std::vector<bool> need(n * n, false);
    for (auto &d : info.dens)
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j)
                if ((d.mask >> i & 1) && (d.mask >> j & 1)) need[i * n + j] = true;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (need[i * n + j]) {
                // 2 P_i . P_j with P = momentum into the diagram (sign of the leg)
                double sg = (p.leg_incoming[i] ? 1.0 : -1.0) * (p.leg_incoming[j] ? 1.0 : -1.0);
                o << "  const T d" << i << "_" << j << " = " << (sg > 0 ? "" : "-")
                  << "2.0 * (p[" << i << "][0] * p[" << j << "][0] - p[" << i << "][1] * p[" << j
                  << "][1] - p[" << i << "][2] * p[" << j << "][2] - p[" << i << "][3] * p[" << j
                  << "][3]);\n";
            }
    for (int s = 0; s < info.n_den; ++s) {
        const DenSlot &d = info.dens[s];
        // P^2 - M^2 = (sum of the legs' m^2 - M^2) + sum of 2 P_i.P_j: the mass
        // terms first, so that an on-shell mass cancels exactly before the
        // (possibly small) invariants are added
        o << "  den[" << s << "] = (T(0.0)";
        for (int i = 0; i < n; ++i)
            if ((d.mask >> i & 1) && p.leg_mass_id[i] >= 0)
                o << " + masses[" << p.leg_mass_id[i] << "] * masses[" << p.leg_mass_id[i] << "]";
        if (d.mass_id >= 0) o << " - masses[" << d.mass_id << "] * masses[" << d.mass_id << "]";
        o << ")";
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j)
                if ((d.mask >> i & 1) && (d.mask >> j & 1)) o << " + d" << i << "_" << j;
        o << ";\n";
    }
    o << "}\n";
}

std::string generate_source(const mf_process &p, int precision, int block, int ht, GenInfo &info, const char *ns,
                            bool kernel, int min_blocks) {
    const char *R = precision == MF_FP64 ? "double" : "float";
    const int n = p.n_legs;
    std::ostringstream o;
    std::vector<uint32_t> mask;
    emit_header(o, p, info, mask, R, ns);
    // The vertex routines are called as non-inlined functions: one copy of each
    // routine's code instead of one per use.  A long program then fits the
    // instruction caches far better (the inlined form is fetch-bound), at the
    // price of argument passing: long programs call every routine (mode 1),
    // shorter ones inline the currents and call the amplitude routines
    // (mode 3; gg -> tt~g 1.12x faster than mode 1).  The process option
    // call_routines overrides: 0 inlines everything, 2 calls the currents only.
    int call_mode = large_program(p) ? 1 : 3;
    if (p.opt.call_routines >= 0) call_mode = p.opt.call_routines;
    const bool calls = call_mode != 0;
    auto rt = [&](const char *name) {
        const bool amp = std::string(name).find("_AMP") != std::string::npos;
        const bool call = call_mode == 1 || (call_mode == 2 && !amp) || (call_mode == 3 && amp);
        return std::string(call ? "n" : "") + name;
    };
    auto a4r = [&](const char *routine, const char *name) {
        std::string n(name);
        if (rt(routine)[0] != 'n') return n;
        return n + "[0], " + n + "[1], " + n + "[2], " + n + "[3]";
    };

    // --- the program for one helicity
    // momentum into the diagram through the legs of a mask, component q
    auto mom = [&](uint32_t m, const std::string &name) {
        std::ostringstream e;
        e << "    const R " << name << "[4] = {";
        for (int q = 0; q < 4; ++q) {
            bool first = true;
            for (int l = 0; l < n; ++l)
                if (m >> l & 1) {
                    bool plus = p.leg_incoming[l] != 0;
                    e << (first ? (plus ? "" : "-") : (plus ? " + " : " - ")) << "ms[" << 4 * l + q << "]";
                    first = false;
                }
            e << (q < 3 ? ", " : "};\n");
        }
        return e.str();
    };
    // amplitude order: greedy over the amplitude units, the unit needing the
    // fewest wavefunctions not yet computed first (ties: the one releasing
    // most live values), which keeps the number of live wavefunctions small
    const std::vector<AmpUnit> units = amplitude_units(p);
    std::function<void(int, std::vector<char> &)> closure = [&](int k, std::vector<char> &seen) {
        for (int q = 0; q < 4; ++q) {
            int i = p.ops[k].in[q];
            if (i >= 0 && !seen[i]) { seen[i] = 1; closure(i, seen); }
        }
    };
    std::vector<std::vector<int>> need_wf(units.size());
    for (size_t u = 0; u < units.size(); ++u) {
        std::vector<char> seen(p.ops.size(), 0);
        for (int a : units[u].ops) closure(a, seen);
        for (size_t i = 0; i < seen.size(); ++i)
            if (seen[i]) need_wf[u].push_back((int)i);
    }
    std::vector<int> uses(p.ops.size(), 0);
    for (auto &op : p.ops)
        for (int q = 0; q < 4; ++q)
            if (op.in[q] >= 0) uses[op.in[q]]++;
    std::vector<char> done(p.ops.size(), 0);
    std::vector<int> remaining_uses = uses;
    std::vector<int> order;               // unit indices
    std::vector<char> taken(units.size(), 0);
    for (size_t step = 0; step < units.size(); ++step) {
        int best = -1, bnew = 0, bfree = 0;
        for (size_t u = 0; u < units.size(); ++u) {
            if (taken[u]) continue;
            int nnew = 0;
            for (int i : need_wf[u]) nnew += !done[i];
            std::map<int, int> used;
            for (int a : units[u].ops)
                for (int q = 0; q < 4; ++q)
                    if (p.ops[a].in[q] >= 0) used[p.ops[a].in[q]]++;
            int nfree = 0;
            for (auto &e : used)
                if (done[e.first] && remaining_uses[e.first] == e.second) ++nfree;
            if (best < 0 || nnew < bnew || (nnew == bnew && nfree > bfree)) { best = (int)u; bnew = nnew; bfree = nfree; }
        }
        taken[best] = 1;
        order.push_back(best);
        for (int i : need_wf[best])
            if (!done[i]) {
                done[i] = 1;
                for (int q = 0; q < 4; ++q)
                    if (p.ops[i].in[q] >= 0) remaining_uses[p.ops[i].in[q]]--;
            }
        for (int a : units[best].ops)
            for (int q = 0; q < 4; ++q)
                if (p.ops[a].in[q] >= 0) remaining_uses[p.ops[a].in[q]]--;
    }
    // then a local search lowers the peak of live wavefunctions (grouped
    // units need several vector currents at once)
    {
        bool grouped = false;
        for (const AmpUnit &un : units) grouped |= un.ops.size() > 1;
        int iters = grouped ? 4000 : 0;
        if (p.opt.order_search >= 0) iters = p.opt.order_search;
        improve_order(p, units, order, iters);
        info.peak_live = live_profile(p, units, order).first;
    }
    // With inlined routines the schedule is split into parts compiled as
    // separate functions: ptxas falls back to a stack-based allocation for
    // very large functions, so the program is cut into pieces below a size
    // budget; each part recomputes the few shared wavefunctions it needs.
    // Called routines keep the program small enough for twice the budget.
    //
    // Two programs are emitted: one helicity, and a pair of helicities that
    // differ only in the helicity of leg L = pair_leg(p).  In the pair form
    // every wavefunction whose momentum does not flow through leg L is the
    // same for both members and is computed once; the others (and every
    // amplitude) twice, the second copy carrying the suffix _b.
    const int L = pair_leg(p);
    // long programs: a block barrier every 16 amplitudes keeps the block's
    // warps on the same stretch of code, so that the instructions one warp
    // fetched serve the others (measured on gg -> tt~gg: 1.09x)
    int sync_every = large_program(p) ? 16 : 0;
    if (p.opt.sync_every >= 0) sync_every = p.opt.sync_every;
    auto M = [&](int id) { return id >= 0 ? "mass[" + std::to_string(id) + "]" : std::string("R(0)"); };
    // the phase class of coupling c for the routines' products (pmul): 1
    // real, 2 imaginary, 0 general
    auto PH = [&](int c) {
        if (c < 0 || 2 * c + 1 >= (int)p.couplings.size()) return std::string("0");
        const double re = p.couplings[2 * c], im = p.couplings[2 * c + 1];
        return std::to_string(im == 0.0 ? 1 : re == 0.0 ? 2 : 0);
    };
    auto emit_program = [&](const bool pair) {
    auto dep = [&](int k) { return pair && (p.ops[k].kind == MF_OP_AMP || (mask[k] >> L & 1)); };
    auto nm = [&](int k, const char *sfx) { return "w" + std::to_string(k) + (dep(k) ? sfx : ""); };
    double weight = 0.0;
    for (size_t k = 0; k < p.ops.size(); ++k) weight += routine_flops(p.ops[k].routine) * (dep((int)k) ? 2 : 1);
    if (precision == MF_FP64) weight *= 2.0;
    int parts = (int)std::ceil(weight / (calls ? 64000.0 : 32000.0));
    if (p.opt.program_parts >= 1) parts = p.opt.program_parts;
    if (parts < 1) parts = 1;
    if (parts > (int)order.size()) parts = (int)order.size();
    if (!pair) info.parts = parts;
    const std::string fn = pair ? "program_pair_part" : "program_part";
    // one wavefunction (suffix "" or "_b": which member's inputs it takes)
    auto emit_one = [&](int k, const char *sfx) {
        const mf_op &op = p.ops[k];
        const std::string wk = "w" + std::to_string(k) + sfx;
        if (op.kind == MF_OP_EXT) {
            int l = op.leg;
            // leg L of a pair: member a has helicity -1, member b +1
            const std::string h = (pair && l == L) ? (sfx[0] ? "1" : "-1") : "hel[" + std::to_string(l) + "]";
            if (op.routine == MF_R_VXX) {
                o << "  const W<R> " << wk << " = vxx<R>(ms + " << 4 * l << ", " << h << ", "
                  << (p.leg_incoming[l] ? 1 : 0) << ");\n";
            } else {
                // column: u (incoming particle) or v (outgoing antiparticle);
                // row: u-bar (outgoing particle) or v-bar (incoming antiparticle)
                int anti = (op.routine == MF_R_IXX) ? (p.leg_incoming[l] ? 0 : 1) : (p.leg_incoming[l] ? 1 : 0);
                o << "  const W<R> " << wk << " = " << (op.routine == MF_R_IXX ? "ixx" : "oxx") << "<R>(ms + " << 4 * l
                  << ", " << M(p.leg_mass_id[l]) << ", " << h << ", " << anti << ");\n";
            }
            return;
        }
        std::string g = "cpl[" + std::to_string(op.coupling) + "]";
        std::string den = "idn[" + std::to_string(info.op_den[k]) + "]";
        auto in = [&](int q) { return nm(op.in[q], sfx); };
        o << "  W<R> " << wk << ";\n  {\n";
        switch (op.routine) {
            case MF_R_FFV_FIN:
            case MF_R_FFV_FOUT:
                o << mom(mask[k], "P");
                o << "    " << wk << " = " << rt(op.routine == MF_R_FFV_FIN ? "FFV_FIN" : "FFV_FOUT") << "<R, "
                  << PH(op.coupling) << ">("
                  << in(0) << ", " << in(1) << ", " << g << ", " << M(op.mass_id) << ", " << den << ", "
                  << a4r("FFV_FIN", "P") << ");\n";
                break;
            case MF_R_FFV_VEC:
                o << "    " << wk << " = " << rt("FFV_VEC") << "<R, " << PH(op.coupling) << ">(" << in(0) << ", "
                  << in(1) << ", " << g << ", "
                  << den << ");\n";
                break;
            case MF_R_VVV_VEC:
                o << mom(mask[op.in[0]], "kA") << mom(mask[op.in[1]], "kB");
                o << "    " << wk << " = " << rt("VVV_VEC") << "<R, " << PH(op.coupling) << ">(" << in(0) << ", "
                  << in(1) << ", "
                  << a4r("VVV_VEC", "kA") << ", " << a4r("VVV_VEC", "kB") << ", " << g << ", " << den << ");\n";
                break;
            default:
                o << "    " << wk << " = " << rt("VVVV_VEC") << "<R, " << (op.routine - MF_R_VVVV1_VEC + 1) << ", "
                  << PH(op.coupling) << ">("
                  << in(0) << ", " << in(1) << ", " << in(2) << ", " << g << ", " << den << ");\n";
                break;
        }
        o << "  }\n";
    };
    // emission: each wavefunction (both copies in a pair) just before the
    // first amplitude needing it
    std::function<void(int)> emit_wf = [&](int k) {
        if (done[k]) return;
        const mf_op &op = p.ops[k];
        for (int q = 0; q < 4; ++q)
            if (op.in[q] >= 0) emit_wf(op.in[q]);
        done[k] = 1;
        emit_one(k, "");
        if (dep(k)) emit_one(k, "_b");
    };
    // an amplitude's colour coefficients into the flows Jn
    auto emit_terms = [&](const mf_op &op, const std::string &Jn, const std::string &a) {
        for (int t = 0; t < op.n_terms; ++t) {
            const mf_colour_term &ct = p.terms[op.first_term + t];
            std::string Jk = Jn + "[" + std::to_string(ct.jamp) + "]";
            if (ct.im == 0.0 && ct.re == 1.0) o << "    " << Jk << " = " << Jk << " + " << a << ";\n";
            else if (ct.im == 0.0 && ct.re == -1.0) o << "    " << Jk << " = " << Jk << " - " << a << ";\n";
            else if (ct.re == 0.0 && ct.im == 1.0) o << "    " << Jk << " = " << Jk << " + mul_i(" << a << ");\n";
            else if (ct.re == 0.0 && ct.im == -1.0) o << "    " << Jk << " = " << Jk << " - mul_i(" << a << ");\n";
            else
                o << "    " << Jk << " = cfma(C<R>(R(" << fmt_double(ct.re) << "), R(" << fmt_double(ct.im)
                  << ")), " << a << ", " << Jk << ");\n";
        }
    };
    // one amplitude into the colour flows J (member a) or Jb (member b)
    auto emit_amp = [&](int k, const char *sfx) {
        const mf_op &op = p.ops[k];
        auto in = [&](int q) { return nm(op.in[q], sfx); };
        std::string g = "cpl[" + std::to_string(op.coupling) + "]";
        const std::string Jn = sfx[0] ? "Jb" : "J";
        o << "  {\n";
        if (op.routine == MF_R_VVV_AMP) o << mom(mask[op.in[0]], "kA") << mom(mask[op.in[1]], "kB") << mom(mask[op.in[2]], "kC");
        o << "    const cx<R> a = ";
        switch (op.routine) {
            case MF_R_FFV_AMP:
                o << rt("FFV_AMP") << "<R, " << PH(op.coupling) << ">(" << in(0) << ", " << in(1) << ", " << in(2)
                  << ", " << g << ")";
                break;
            case MF_R_VVV_AMP:
                o << rt("VVV_AMP") << "<R, " << PH(op.coupling) << ">(" << in(0) << ", " << in(1) << ", " << in(2)
                  << ", "
                  << a4r("VVV_AMP", "kA") << ", " << a4r("VVV_AMP", "kB") << ", " << a4r("VVV_AMP", "kC") << ", " << g
                  << ")";
                break;
            default:
                o << rt("VVVV_AMP") << "<R, " << (op.routine - MF_R_VVVV1_AMP + 1) << ", " << PH(op.coupling) << ">("
                  << in(0) << ", " << in(1)
                  << ", " << in(2) << ", " << in(3) << ", " << g << ")";
        }
        o << ";\n";
        emit_terms(op, Jn, "a");
        o << "  }\n";
    };
    // the two amplitudes of a pair: one call when they differ only in the
    // row or only in the column spinor (the V-slash product shared)
    auto emit_amp_pair = [&](int k) {
        const mf_op &op = p.ops[k];
        int dq = -1, ndep = 0;
        for (int q = 0; q < 4; ++q)
            if (op.in[q] >= 0 && dep(op.in[q])) { dq = q; ++ndep; }
        if (op.routine != MF_R_FFV_AMP || ndep != 1 || dq > 1) {
            emit_amp(k, "");
            emit_amp(k, "_b");
            return;
        }
        std::string g = "cpl[" + std::to_string(op.coupling) + "]";
        const std::string r = rt(dq == 0 ? "FFV_AMP_R2" : "FFV_AMP_C2");
        const std::string v = "w" + std::to_string(op.in[dq]);
        o << "  {\n    const A2<R> ab = " << r << "<R, " << PH(op.coupling) << ">(";
        if (dq == 0) o << v << ", " << v << "_b, w" << op.in[1];
        else o << "w" << op.in[0] << ", " << v << ", " << v << "_b";
        o << ", w" << op.in[2] << ", " << g << ");\n";
        emit_terms(op, "J", "ab.a");
        emit_terms(op, "Jb", "ab.b");
        o << "  }\n";
    };
    // a unit of several FFV amplitudes: their vector currents combined with
    // the members' phases, one amplitude (or one pair of amplitudes), the
    // first member's colour coefficients
    auto emit_unit = [&](const AmpUnit &un) {
        const mf_op &op0 = p.ops[un.ops[0]];
        bool vdep = false;
        for (int a : un.ops) vdep |= dep(p.ops[a].in[2]);
        o << "  {\n";
        auto build = [&](const char *sfx, const std::string &vs) {
            o << "    W<R> " << vs << " = " << nm(op0.in[2], sfx) << ";\n";
            for (size_t m = 1; m < un.ops.size(); ++m) {
                const std::string v = nm(p.ops[un.ops[m]].in[2], sfx) + ".c[c]";
                const int ph = un.phase[m];
                o << "#pragma unroll\n    for (int c = 0; c < 4; ++c) " << vs << ".c[c] = " << vs << ".c[c] "
                  << (ph == 0 ? "+ " + v : ph == 2 ? "- " + v : ph == 1 ? "+ mul_i(" + v + ")" : "- mul_i(" + v + ")")
                  << ";\n";
            }
        };
        build("", "vs");
        if (pair && vdep) build("_b", "vs_b");
        const std::string g = "cpl[" + std::to_string(op0.coupling) + "]";
        const bool rdep = pair && dep(op0.in[0]), cdep = pair && dep(op0.in[1]);
        const std::string row = "w" + std::to_string(op0.in[0]), col = "w" + std::to_string(op0.in[1]);
        if (!pair) {
            o << "    const cx<R> a = " << rt("FFV_AMP") << "<R, " << PH(op0.coupling) << ">(" << row << ", " << col
              << ", vs, " << g << ");\n";
            emit_terms(op0, "J", "a");
        } else if (!vdep && rdep != cdep) {
            o << "    const A2<R> ab = " << rt(rdep ? "FFV_AMP_R2" : "FFV_AMP_C2") << "<R, " << PH(op0.coupling) << ">(";
            if (rdep) o << row << ", " << row << "_b, " << col;
            else o << row << ", " << col << ", " << col << "_b";
            o << ", vs, " << g << ");\n";
            emit_terms(op0, "J", "ab.a");
            emit_terms(op0, "Jb", "ab.b");
        } else {
            o << "    const cx<R> a = " << rt("FFV_AMP") << "<R, " << PH(op0.coupling) << ">(" << row << ", " << col
              << ", vs, " << g << ");\n";
            o << "    const cx<R> b = " << rt("FFV_AMP") << "<R, " << PH(op0.coupling) << ">(" << nm(op0.in[0], "_b")
              << ", " << nm(op0.in[1], "_b")
              << ", " << (vdep ? "vs_b" : "vs") << ", " << g << ");\n";
            emit_terms(op0, "J", "a");
            emit_terms(op0, "Jb", "b");
        }
        o << "  }\n";
    };
    for (int part = 0; part < parts; ++part) {
    std::fill(done.begin(), done.end(), 0);
    const size_t lo = order.size() * part / parts, hi = order.size() * (part + 1) / parts;
    o << "template <typename R>\n" << (parts > 1 ? "__device__ __noinline__" : "MF_DEV") << " void " << fn << part
      << "(const R *__restrict__ ms, const R *__restrict__ idn, const int8_t *__restrict__ hel,\n"
         "    const mf::cx<R> *__restrict__ cpl, const R *__restrict__ mass, mf::cx<R> *__restrict__ Jout"
      << (pair ? ", mf::cx<R> *__restrict__ Jout_b" : "") << ") {\n"
         "  using namespace mf;\n"
         "  cx<R> J[NJAMP];\n#pragma unroll\n  for (int k = 0; k < NJAMP; ++k) J[k] = C<R>(R(0), R(0));\n";
    if (pair) o << "  cx<R> Jb[NJAMP];\n#pragma unroll\n  for (int k = 0; k < NJAMP; ++k) Jb[k] = C<R>(R(0), R(0));\n";
    for (size_t oi = lo; oi < hi; ++oi) {
        const AmpUnit &un = units[order[oi]];
        // keep the block's warps on the same stretch of code, so that fetched
        // instructions serve all of them
        if (sync_every > 0 && oi > lo && (oi - lo) % sync_every == 0) o << "  MF_PROG_SYNC();\n";
        for (int a : un.ops)
            for (int q = 0; q < 4; ++q)
                if (p.ops[a].in[q] >= 0) emit_wf(p.ops[a].in[q]);
        if (un.ops.size() > 1) emit_unit(un);
        else if (pair) emit_amp_pair(un.ops[0]);
        else emit_amp(un.ops[0], "");
    }
    o << "#pragma unroll\n  for (int k = 0; k < NJAMP; ++k) Jout[k] = Jout[k] + J[k];\n";
    if (pair) o << "#pragma unroll\n  for (int k = 0; k < NJAMP; ++k) Jout_b[k] = Jout_b[k] + Jb[k];\n";
    o << "}\n";
    }
    return parts;
    };
    const int parts = emit_program(false);
    const int pair_parts = L >= 0 ? emit_program(true) : 0;
    // colour sum  sum_kl Re(conj(J_k) C_kl J_l) / den, C symmetric:
    // sum_k Re(conj(J_k) (C_kk J_k + 2 sum_{l>k} C_kl J_l))
    const int nj = p.n_jamp;
    o << "template <typename R>\nMF_DEV R colour_sum_full(const mf::cx<R> *J) {\n  using namespace mf;\n  R m = R(0);\n";
    for (int k = 0; k < nj; ++k) {
        o << "  { cx<R> z = R(" << p.colour_num[k * nj + k] << ") * J[" << k << "];\n";
        for (int l = k + 1; l < nj; ++l) {
            int c = p.colour_num[k * nj + l];
            if (c == 0) continue;
            o << "    z = z + R(" << 2 * c << ") * J[" << l << "];\n";
        }
        o << "    m += J[" << k << "].re * z.re + J[" << k << "].im * z.im; }\n";
    }
    o << "  return m * R(" << fmt_double(1.0 / p.colour_den) << ");\n}\n";
    // leading colour: the diagonal of the colour matrix in the flow basis
    o << "template <typename R>\nMF_DEV R colour_sum_lc(const mf::cx<R> *J) {\n  using namespace mf;\n  R m = R(0);\n";
    for (int k = 0; k < nj; ++k)
        o << "  m += R(" << p.colour_num[k * nj + k] << ") * (J[" << k << "].re * J[" << k << "].re + J[" << k
          << "].im * J[" << k << "].im);\n";
    o << "  return m * R(" << fmt_double(1.0 / p.colour_den) << ");\n}\n";
    o << "template <typename R>\n"
         "MF_DEV R helicity_msq(const R *__restrict__ ms, const R *__restrict__ idn, const int8_t *hel,\n"
         "                      const mf::cx<R> *cpl, const R *mass) {\n"
         "  using namespace mf;\n"
         "  cx<R> J[NJAMP];\n#pragma unroll\n  for (int k = 0; k < NJAMP; ++k) J[k] = C<R>(R(0), R(0));\n";
    for (int part = 0; part < parts; ++part) o << "  program_part" << part << "<R>(ms, idn, hel, cpl, mass, J);\n";
    o << "  return colour_sum_full<R>(J);\n}\n";
    // the colour flows alone (the colour sum done by the caller), the colour
    // matrix's integer numerators and the inverse denominator
    o << "template <typename R>\n"
         "MF_DEV void helicity_jamp(const R *__restrict__ ms, const R *__restrict__ idn, const int8_t *hel,\n"
         "                          const mf::cx<R> *cpl, const R *mass, mf::cx<R> *J) {\n"
         "  using namespace mf;\n#pragma unroll\n  for (int k = 0; k < NJAMP; ++k) J[k] = C<R>(R(0), R(0));\n";
    for (int part = 0; part < parts; ++part) o << "  program_part" << part << "<R>(ms, idn, hel, cpl, mass, J);\n";
    o << "}\n";
    // a pair of helicities (the kernel's row with leg PAIR_LEG at -1, then at
    // +1): both colour-summed |M|^2
    o << "constexpr int PAIR_LEG = " << L << ";\n"
         "template <typename R>\n"
         "MF_DEV void helicity_pair_msq(const R *__restrict__ ms, const R *__restrict__ idn, const int8_t *hel,\n"
         "                              const mf::cx<R> *cpl, const R *mass, R &va, R &vb) {\n"
         "  using namespace mf;\n";
    if (L >= 0) {
        o << "  cx<R> J[NJAMP], Jb[NJAMP];\n#pragma unroll\n"
             "  for (int k = 0; k < NJAMP; ++k) { J[k] = C<R>(R(0), R(0)); Jb[k] = J[k]; }\n";
        for (int part = 0; part < pair_parts; ++part)
            o << "  program_pair_part" << part << "<R>(ms, idn, hel, cpl, mass, J, Jb);\n";
        o << "  if constexpr (LEADING_COLOUR) { va = colour_sum_lc<R>(J); vb = colour_sum_lc<R>(Jb); }\n"
             "  else { va = colour_sum_full<R>(J); vb = colour_sum_full<R>(Jb); }\n";
    } else {
        o << "  va = vb = R(0);\n";
    }
    o << "}\n";
    // the colour flows of a helicity pair without their colour sums
    o << "template <typename R>\n"
         "MF_DEV void helicity_pair_jamp(const R *__restrict__ ms, const R *__restrict__ idn, const int8_t *hel,\n"
         "                               const mf::cx<R> *cpl, const R *mass, mf::cx<R> *J, mf::cx<R> *Jb) {\n"
         "  using namespace mf;\n#pragma unroll\n"
         "  for (int k = 0; k < NJAMP; ++k) { J[k] = C<R>(R(0), R(0)); Jb[k] = J[k]; }\n";
    for (int part = 0; part < pair_parts; ++part)
        o << "  program_pair_part" << part << "<R>(ms, idn, hel, cpl, mass, J, Jb);\n";
    o << "}\n__device__ const int COLOUR_NUM[NJAMP * NJAMP] = {";
    for (int k = 0; k < nj * nj; ++k) o << (k ? ", " : "") << p.colour_num[k];
    o << "};\nconstexpr double INV_COLOUR_DEN = " << fmt_double(1.0 / p.colour_den) << ";\n";
    // one row of the colour sum: Re(conj(J_k) sum_l C_kl J_l) (numerators),
    // k chosen at run time (selected, not indexed, so J stays in registers)
    o << "template <typename R>\nMF_DEV R colour_row(const mf::cx<R> *J, int k) {\n  using namespace mf;\n"
         "  cx<R> jk = C<R>(R(0), R(0)), z = jk;\n#pragma unroll\n"
         "  for (int l = 0; l < NJAMP; ++l) {\n    if (l == k) jk = J[l];\n"
         "    z = z + R(COLOUR_NUM[k * NJAMP + l]) * J[l];\n  }\n"
         "  return jk.re * z.re + jk.im * z.im;\n}\n";
    o << "}  // namespace " << ns << "\n";
    if (kernel) {
        o << "#include \"mf_kernel.cuh\"\n";
        // optional minimum of resident blocks per SM (trades registers for occupancy)
        if (min_blocks < 0) min_blocks = p.opt.min_blocks > 0 ? p.opt.min_blocks : 0;
        o << "extern \"C\" __global__ void __launch_bounds__(" << block;
        if (min_blocks >= 1 && min_blocks <= 8) o << ", " << min_blocks;
        o << ") mf_kernel(const mf::KParams kp) {\n";
        if (precision == MF_MIXED_TC) o << "  mf::kernel_body_tc<" << ht << ">(kp);\n}\n";
        else o << "  mf::kernel_body<" << R << ", " << block << ", " << ht << ">(kp);\n}\n";
        // the leading-colour flow kernel (mode 5) and the colour-sampled
        // integrand kernel of the same programs
        const int fblock = precision == MF_MIXED_TC ? 128 : block;
        o << "extern \"C\" __global__ void __launch_bounds__(" << fblock << ") mf_flow_kernel(const mf::KParams kp) {\n"
          << "  mf::kernel_body<" << R << ", " << fblock << ", " << ht << ", 1>(kp);\n}\n";
        o << "extern \"C\" __global__ void __launch_bounds__(" << fblock << ") mf_csamp_kernel(const mf::KParams kp) {\n"
          << "  mf::kernel_body<" << R << ", " << fblock << ", " << ht << ", 2>(kp);\n}\n";
    }
    // algorithmic count of the programs as emitted: every wavefunction once
    // (the few a later program part recomputes are not counted), per
    // amplitude unit one amplitude, the combination of its vector currents
    // (a complex add per component and extra member) and the first member's
    // colour coefficients, and the colour sum
    double alg = 0.0;
    for (const mf_op &op : p.ops)
        if (op.kind != MF_OP_AMP) alg += op_flops(p, op);
    for (const AmpUnit &un : units) {
        const mf_op &op0 = p.ops[un.ops[0]];
        alg += op_flops(p, op0) + 8.0 * (un.ops.size() - 1) + term_flops(p, op0);
    }
    alg += colour_sum_flops(p);
    info.flops_per_hel = alg;
    info.pair_leg = L;
    // the pair program: wavefunctions independent of leg L once, the others
    // twice; per unit the combination once or (vector currents depending on
    // L) twice, and one shared V-slash product with two spinor products (136
    // FLOPs) where only the row or only the column spinor differs, else two
    // amplitudes; both members' colour coefficients and colour sums
    info.flops_pair = 0.0;
    if (L >= 0) {
        double fp = 0.0;
        auto dep_wf = [&](int i) { return p.ops[i].kind != MF_OP_AMP && (mask[i] >> L & 1); };
        for (size_t k = 0; k < p.ops.size(); ++k)
            if (p.ops[k].kind != MF_OP_AMP) fp += op_flops(p, p.ops[k]) * (dep_wf((int)k) ? 2 : 1);
        for (const AmpUnit &un : units) {
            const mf_op &op0 = p.ops[un.ops[0]];
            bool vdep = false;
            for (int a : un.ops) vdep |= op0.routine == MF_R_FFV_AMP && dep_wf(p.ops[a].in[2]);
            fp += 8.0 * (un.ops.size() - 1) * (vdep ? 2 : 1);
            bool shared;
            if (un.ops.size() > 1) {
                shared = !vdep && (dep_wf(op0.in[0]) != dep_wf(op0.in[1]));
            } else {
                int ndep = 0, dq = -1;
                for (int q = 0; q < 4; ++q)
                    if (op0.in[q] >= 0 && dep_wf(op0.in[q])) { ++ndep; dq = q; }
                shared = op0.routine == MF_R_FFV_AMP && ndep == 1 && dq <= 1;
            }
            // (the shared form's two products with the coupling: 2 x 4 FLOPs
            // fewer for a real or imaginary coupling, as op_flops)
            fp += shared ? 136.0 - 2.0 * (routine_flops(op0.routine) - op_flops(p, op0)) : 2.0 * op_flops(p, op0);
            fp += 2.0 * term_flops(p, op0);
        }
        fp += 2.0 * colour_sum_flops(p);
        info.flops_pair = fp;
    }
    // kinematics per event (phase space, PDFs, denominators), rough count
    info.flops_kin = 400.0 + 10.0 * info.n_den;
    return o.str();
}


// Momentum into the diagram through the legs of a mask, as a local array.
static std::string mom_array(const mf_process &p, uint32_t m, const std::string &name) {
    std::ostringstream e;
    e << "    const R " << name << "[4] = {";
    for (int q = 0; q < 4; ++q) {
        bool first = true;
        for (int l = 0; l < p.n_legs; ++l)
            if (m >> l & 1) {
                bool plus = p.leg_incoming[l] != 0;
                e << (first ? (plus ? "" : "-") : (plus ? " + " : " - ")) << "ms[" << 4 * l + q << "]";
                first = false;
            }
        e << (q < 3 ? ", " : "};\n");
    }
    return e.str();
}

// Adjoint of a momentum (array name) spread over the external legs of a mask.
static std::string mom_scatter(const mf_process &p, uint32_t m, const std::string &name) {
    std::ostringstream e;
    for (int l = 0; l < p.n_legs; ++l)
        if (m >> l & 1)
            for (int q = 0; q < 4; ++q)
                e << "    pbar[" << 4 * l + q << "] " << (p.leg_incoming[l] ? "+=" : "-=") << " " << name << "[" << q
                  << "];\n";
    return e.str();
}

std::string generate_grad_source(const mf_process &p, int block, GenInfo &info) {
    std::ostringstream o;
    std::vector<uint32_t> mask;
    o << "#include \"mf_helas_adj.cuh\"\n";
    emit_header(o, p, info, mask, "double");
    // compact indices of the wavefunctions
    std::vector<int> ci(p.ops.size(), -1);
    int nwf = 0;
    for (size_t k = 0; k < p.ops.size(); ++k)
        if (p.ops[k].kind != MF_OP_AMP) ci[k] = nwf++;
    auto W_ = [&](int k) { return "w[" + std::to_string(ci[k]) + "]"; };
    auto WB = [&](int k) { return "wb[" + std::to_string(ci[k]) + "]"; };
    auto M = [&](int id) { return id >= 0 ? "mass[" + std::to_string(id) + "]" : std::string("R(0)"); };
    o << "template <typename R>\nMF_DEV R helicity_msq(const R *, const R *, const int8_t *, const mf::cx<R> *, const R *);\n";
    // The program is emitted as many small non-inlined functions sharing the
    // wavefunction arrays through pointers: one large function would fall
    // into ptxas's low-quality allocation and compile slowly.
    const int CH = 12;
    const char *args =
        "(const R *__restrict__ ms, const R *__restrict__ idn, const int8_t *__restrict__ hel, "
        "const mf::cx<R> *__restrict__ cpl, const R *__restrict__ mass, mf::W<R> *__restrict__ w, "
        "mf::W<R> *__restrict__ wb, mf::cx<R> *__restrict__ J, mf::cx<R> *__restrict__ Jb, R *__restrict__ pbar, "
        "R *__restrict__ idnbar, R *__restrict__ mbar)";
    std::vector<std::string> calls;
    int nfun = 0;
    auto open_fn = [&]() {
        std::string name = "gchunk" + std::to_string(nfun++);
        o << "template <typename R>\n__device__ __noinline__ void " << name << args << " {\n  using namespace mf;\n";
        calls.push_back(name);
    };
    auto close_fn = [&]() { o << "}\n"; };
    // forward sweep (wavefunctions), in op order
    {
        int cnt = 0;
        for (size_t k = 0; k < p.ops.size(); ++k) {
            const mf_op &op = p.ops[k];
            if (op.kind == MF_OP_AMP) continue;
            if (cnt % CH == 0) { if (cnt) close_fn(); open_fn(); }
            ++cnt;
            if (op.kind == MF_OP_EXT) {
                int l = op.leg;
                if (op.routine == MF_R_VXX)
                    o << "  " << W_(k) << " = vxx<R>(ms + " << 4 * l << ", hel[" << l << "], "
                      << (p.leg_incoming[l] ? 1 : 0) << ");\n";
                else {
                    int anti = (op.routine == MF_R_IXX) ? (p.leg_incoming[l] ? 0 : 1) : (p.leg_incoming[l] ? 1 : 0);
                    o << "  " << W_(k) << " = " << (op.routine == MF_R_IXX ? "ixx" : "oxx") << "<R>(ms + " << 4 * l
                      << ", " << M(p.leg_mass_id[l]) << ", hel[" << l << "], " << anti << ");\n";
                }
                continue;
            }
            std::string g = "cpl[" + std::to_string(op.coupling) + "]";
            std::string den = "idn[" + std::to_string(info.op_den[k]) + "]";
            o << "  {\n";
            switch (op.routine) {
                case MF_R_FFV_FIN: case MF_R_FFV_FOUT:
                    o << mom_array(p, mask[k], "P") << "    " << W_(k) << " = "
                      << (op.routine == MF_R_FFV_FIN ? "FFV_FIN" : "FFV_FOUT") << "<R>(" << W_(op.in[0]) << ", "
                      << W_(op.in[1]) << ", " << g << ", " << M(op.mass_id) << ", " << den << ", P);\n";
                    break;
                case MF_R_FFV_VEC:
                    o << "    " << W_(k) << " = FFV_VEC<R>(" << W_(op.in[0]) << ", " << W_(op.in[1]) << ", " << g
                      << ", " << den << ");\n";
                    break;
                case MF_R_VVV_VEC:
                    o << mom_array(p, mask[op.in[0]], "kA") << mom_array(p, mask[op.in[1]], "kB") << "    " << W_(k)
                      << " = VVV_VEC<R>(" << W_(op.in[0]) << ", " << W_(op.in[1]) << ", kA, kB, " << g << ", " << den
                      << ");\n";
                    break;
                default:
                    o << "    " << W_(k) << " = VVVV_VEC<R, " << (op.routine - MF_R_VVVV1_VEC + 1) << ">("
                      << W_(op.in[0]) << ", " << W_(op.in[1]) << ", " << W_(op.in[2]) << ", " << g << ", " << den
                      << ");\n";
            }
            o << "  }\n";
        }
        if (cnt) close_fn();
    }
    // amplitudes -> colour flows
    std::vector<int> amps;
    for (size_t k = 0; k < p.ops.size(); ++k)
        if (p.ops[k].kind == MF_OP_AMP) amps.push_back((int)k);
    for (size_t a = 0; a < amps.size(); ++a) {
        if (a % CH == 0) { if (a) close_fn(); open_fn(); }
        const mf_op &op = p.ops[amps[a]];
        std::string g = "cpl[" + std::to_string(op.coupling) + "]";
        o << "  {\n";
        if (op.routine == MF_R_VVV_AMP)
            o << mom_array(p, mask[op.in[0]], "kA") << mom_array(p, mask[op.in[1]], "kB") << mom_array(p, mask[op.in[2]], "kC");
        o << "    const cx<R> a = ";
        switch (op.routine) {
            case MF_R_FFV_AMP: o << "FFV_AMP<R>(" << W_(op.in[0]) << ", " << W_(op.in[1]) << ", " << W_(op.in[2]) << ", " << g << ")"; break;
            case MF_R_VVV_AMP: o << "VVV_AMP<R>(" << W_(op.in[0]) << ", " << W_(op.in[1]) << ", " << W_(op.in[2]) << ", kA, kB, kC, " << g << ")"; break;
            default:
                o << "VVVV_AMP<R, " << (op.routine - MF_R_VVVV1_AMP + 1) << ">(" << W_(op.in[0]) << ", " << W_(op.in[1])
                  << ", " << W_(op.in[2]) << ", " << W_(op.in[3]) << ", " << g << ")";
        }
        o << ";\n";
        for (int t = 0; t < op.n_terms; ++t) {
            const mf_colour_term &ct = p.terms[op.first_term + t];
            o << "    J[" << ct.jamp << "] = cfma(C<R>(R(" << fmt_double(ct.re) << "), R(" << fmt_double(ct.im)
              << ")), a, J[" << ct.jamp << "]);\n";
        }
        o << "  }\n";
    }
    if (!amps.empty()) close_fn();
    const size_t n_forward = calls.size();
    // adjoints of the amplitudes
    for (size_t a = 0; a < amps.size(); ++a) {
        if (a % CH == 0) { if (a) close_fn(); open_fn(); }
        const mf_op &op = p.ops[amps[a]];
        std::string g = "cpl[" + std::to_string(op.coupling) + "]";
        o << "  {\n    cx<R> ab = C<R>(R(0), R(0));\n";
        for (int t = 0; t < op.n_terms; ++t) {
            const mf_colour_term &ct = p.terms[op.first_term + t];
            o << "    ab = ab + conj(C<R>(R(" << fmt_double(ct.re) << "), R(" << fmt_double(ct.im) << "))) * Jb["
              << ct.jamp << "];\n";
        }
        switch (op.routine) {
            case MF_R_FFV_AMP:
                o << "    FFV_AMP_adj<R>(" << W_(op.in[0]) << ", " << W_(op.in[1]) << ", " << W_(op.in[2]) << ", " << g
                  << ", ab, " << WB(op.in[0]) << ", " << WB(op.in[1]) << ", " << WB(op.in[2]) << ");\n";
                break;
            case MF_R_VVV_AMP:
                o << mom_array(p, mask[op.in[0]], "kA") << mom_array(p, mask[op.in[1]], "kB")
                  << mom_array(p, mask[op.in[2]], "kC")
                  << "    R kAb[4] = {R(0), R(0), R(0), R(0)}, kBb[4] = {R(0), R(0), R(0), R(0)}, kCb[4] = {R(0), R(0), R(0), R(0)};\n"
                  << "    VVV_AMP_adj<R>(" << W_(op.in[0]) << ", " << W_(op.in[1]) << ", " << W_(op.in[2])
                  << ", kA, kB, kC, " << g << ", ab, " << WB(op.in[0]) << ", " << WB(op.in[1]) << ", " << WB(op.in[2])
                  << ", kAb, kBb, kCb);\n"
                  << mom_scatter(p, mask[op.in[0]], "kAb") << mom_scatter(p, mask[op.in[1]], "kBb")
                  << mom_scatter(p, mask[op.in[2]], "kCb");
                break;
            default:
                o << "    VVVV_AMP_adj<R, " << (op.routine - MF_R_VVVV1_AMP + 1) << ">(" << W_(op.in[0]) << ", "
                  << W_(op.in[1]) << ", " << W_(op.in[2]) << ", " << W_(op.in[3]) << ", " << g << ", ab, "
                  << WB(op.in[0]) << ", " << WB(op.in[1]) << ", " << WB(op.in[2]) << ", " << WB(op.in[3]) << ");\n";
        }
        o << "  }\n";
    }
    if (!amps.empty()) close_fn();
    // adjoints of the currents, last first
    {
        int cnt = 0;
        for (size_t kk = p.ops.size(); kk-- > 0;) {
            const mf_op &op = p.ops[kk];
            const int k = (int)kk;
            if (op.kind != MF_OP_CUR) continue;
            if (cnt % CH == 0) { if (cnt) close_fn(); open_fn(); }
            ++cnt;
            std::string g = "cpl[" + std::to_string(op.coupling) + "]";
            int sl = info.op_den[k];
            std::string den = "idn[" + std::to_string(sl) + "]", denb = "idnbar[" + std::to_string(sl) + "]";
            o << "  {\n";
            switch (op.routine) {
                case MF_R_FFV_FIN: case MF_R_FFV_FOUT:
                    o << mom_array(p, mask[k], "P") << "    R Pb[4] = {R(0), R(0), R(0), R(0)}, Mb = R(0);\n    "
                      << (op.routine == MF_R_FFV_FIN ? "FFV_FIN_adj" : "FFV_FOUT_adj") << "<R>(" << W_(op.in[0]) << ", "
                      << W_(op.in[1]) << ", " << g << ", " << M(op.mass_id) << ", " << den << ", P, " << WB(k) << ", "
                      << WB(op.in[0]) << ", " << WB(op.in[1]) << ", " << denb << ", Pb, Mb);\n" << mom_scatter(p, mask[k], "Pb");
                    if (op.mass_id >= 0) o << "    mbar[" << op.mass_id << "] += Mb;\n";
                    break;
                case MF_R_FFV_VEC:
                    o << "    FFV_VEC_adj<R>(" << W_(op.in[0]) << ", " << W_(op.in[1]) << ", " << g << ", " << den << ", "
                      << WB(k) << ", " << WB(op.in[0]) << ", " << WB(op.in[1]) << ", " << denb << ");\n";
                    break;
                case MF_R_VVV_VEC:
                    o << mom_array(p, mask[op.in[0]], "kA") << mom_array(p, mask[op.in[1]], "kB")
                      << "    R kAb[4] = {R(0), R(0), R(0), R(0)}, kBb[4] = {R(0), R(0), R(0), R(0)};\n"
                      << "    VVV_VEC_adj<R>(" << W_(op.in[0]) << ", " << W_(op.in[1]) << ", kA, kB, " << g << ", " << den
                      << ", " << WB(k) << ", " << WB(op.in[0]) << ", " << WB(op.in[1]) << ", " << denb << ", kAb, kBb);\n"
                      << mom_scatter(p, mask[op.in[0]], "kAb") << mom_scatter(p, mask[op.in[1]], "kBb");
                    break;
                default:
                    o << "    VVVV_VEC_adj<R, " << (op.routine - MF_R_VVVV1_VEC + 1) << ">(" << W_(op.in[0]) << ", "
                      << W_(op.in[1]) << ", " << W_(op.in[2]) << ", " << g << ", " << den << ", " << WB(k) << ", "
                      << WB(op.in[0]) << ", " << WB(op.in[1]) << ", " << WB(op.in[2]) << ", " << denb << ");\n";
            }
            o << "  }\n";
        }
        if (cnt) close_fn();
    }
    // external legs: tangents of the wavefunction in its momentum and mass
    {
        int cnt = 0;
        for (size_t k = 0; k < p.ops.size(); ++k) {
            const mf_op &op = p.ops[k];
            if (op.kind != MF_OP_EXT) continue;
            if (cnt % 2 == 0) { if (cnt) close_fn(); open_fn(); }
            ++cnt;
            int l = op.leg;
            int mid = p.leg_mass_id[l];
            std::string mv = mid >= 0 ? "mass[" + std::to_string(mid) + "]" : std::string("R(0)");
            o << "  {\n    R mdummy = R(0);\n    external_adj([&](const Dual<5> *pd, const Dual<5> &md) { return ";
            if (op.routine == MF_R_VXX)
                o << "vxx<Dual<5>>(pd, hel[" << l << "], " << (p.leg_incoming[l] ? 1 : 0) << ");";
            else {
                int anti = (op.routine == MF_R_IXX) ? (p.leg_incoming[l] ? 0 : 1) : (p.leg_incoming[l] ? 1 : 0);
                o << (op.routine == MF_R_IXX ? "ixx" : "oxx") << "<Dual<5>>(pd, md, hel[" << l << "], " << anti << ");";
            }
            o << " }, ms + " << 4 * l << ", " << mv << ", " << WB(k) << ", pbar + " << 4 * l << ", "
              << (mid >= 0 ? "mbar[" + std::to_string(mid) + "]" : std::string("mdummy")) << ");\n  }\n";
        }
        if (cnt) close_fn();
    }
    // driver: forward, |M|^2 and dL/dJ = 2 C J / den, then the adjoint chunks
    const int nj = p.n_jamp;
    o << "template <typename R>\n"
         "MF_DEV R helicity_grad(const R *__restrict__ ms, const R *__restrict__ idn, const int8_t *hel,\n"
         "    const mf::cx<R> *cpl, const R *mass, R *pbar, R *idnbar, R *mbar) {\n"
         "  using namespace mf;\n"
         "  W<R> w[" << nwf << "], wb[" << nwf << "];\n  cx<R> J[NJAMP], Jb[NJAMP];\n"
         "  for (int k = 0; k < NJAMP; ++k) J[k] = C<R>(R(0), R(0));\n";
    for (size_t c = 0; c < n_forward; ++c)
        o << "  " << calls[c] << "<R>(ms, idn, hel, cpl, mass, w, wb, J, Jb, pbar, idnbar, mbar);\n";
    o << "  R m = R(0);\n";
    for (int k = 0; k < nj; ++k) {
        o << "  { cx<R> z = C<R>(R(0), R(0));\n";
        for (int l = 0; l < nj; ++l) {
            int c = p.colour_num[k * nj + l];
            if (c) o << "    z = z + R(" << c << ") * J[" << l << "];\n";
        }
        o << "    m += J[" << k << "].re * z.re + J[" << k << "].im * z.im;\n"
          << "    Jb[" << k << "] = R(" << fmt_double(2.0 / p.colour_den) << ") * z; }\n";
    }
    o << "  m *= R(" << fmt_double(1.0 / p.colour_den) << ");\n";
    o << "  for (int i = 0; i < " << nwf << "; ++i) for (int c = 0; c < 4; ++c) wb[i].c[c] = C<R>(R(0), R(0));\n";
    for (size_t c = n_forward; c < calls.size(); ++c)
        o << "  " << calls[c] << "<R>(ms, idn, hel, cpl, mass, w, wb, J, Jb, pbar, idnbar, mbar);\n";
    o << "  return m;\n}\n}  // namespace proc\n";
    o << "#include \"mf_grad.cuh\"\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << block << ") mf_grad_kernel(const mf::KParams kp) {\n"
      << "  mf::grad_body<proc::NDIM + 1>(kp);\n}\n";
    return o.str();
}

// Several processes in one module: each process's program in its own
// namespace proc<k> with the tile body instantiated for it in body<k>, and one
// persistent kernel in which every block takes the next work item of the
// batch from a global counter (a group of tiles of one process, items of the
// costliest process first) and runs it with that process's code.
std::string generate_batch_source(const std::vector<const mf_process *> &ps, int precision, int block,
                                  const std::vector<int> &hts, std::vector<GenInfo> &infos) {
    const char *R = precision == MF_FP64 ? "double" : "float";
    std::ostringstream o;
    infos.assign(ps.size(), GenInfo{});
    int maxdim = 1;
    for (size_t k = 0; k < ps.size(); ++k) {
        const std::string ns = "proc" + std::to_string(k);
        o << generate_source(*ps[k], precision, block, hts[k], infos[k], ns.c_str(), false);
        o << "#define MF_PROC proc" << k << "\n#define MF_BODY body" << k << "\n#include \"mf_kernel.cuh\"\n";
        maxdim = std::max(maxdim, ps[k]->ndim);
    }
    o << "extern \"C\" __global__ void __launch_bounds__(" << block << ") mf_batch_kernel(const mf_batch_params bp) {\n"
      << "  extern __shared__ __align__(16) unsigned char smem_raw[];\n"
      << "  __shared__ double s_grid[" << maxdim * 65 << "];\n"
      << "  __shared__ mf::cx<" << R << "> cpl[8];\n"
      << "  __shared__ " << R << " mass_r[8];\n"
      << "  __shared__ long long s_item;\n"
      << "  {\n    size_t need = 0;\n";
    for (size_t k = 0; k < ps.size(); ++k)
        o << "    if (body" << k << "::tile_smem_bytes<" << R << ", " << block << ">() > need) need = body" << k
          << "::tile_smem_bytes<" << R << ", " << block << ">();\n";
    o << "    uint32_t have;\n    asm(\"mov.u32 %0, %%dynamic_smem_size;\" : \"=r\"(have));\n"
      << "    if (have < need) {\n"
      << "      if (threadIdx.x == 0) for (int k = 0; k < bp.nproc; ++k) if (bp.kp[k].err) atomicExch(bp.kp[k].err, 2);\n"
      << "      return;\n    }\n  }\n"
      << "  int cur = -1;\n"
      << "  for (;;) {\n"
      << "    __syncthreads();\n"
      << "    if (threadIdx.x == 0) s_item = (long long)atomicAdd((unsigned long long *)bp.counter, 1ull);\n"
      << "    __syncthreads();\n"
      << "    const long long item = s_item;\n"
      << "    if (item >= bp.start[bp.nproc]) break;\n"
      << "    int k = 0;\n"
      << "    while (k + 1 < bp.nproc && item >= bp.start[k + 1]) ++k;\n"
      << "    if (k != cur) {\n"
      << "      switch (k) {\n";
    for (size_t k = 0; k < ps.size(); ++k)
        o << "        case " << k << ": body" << k << "::load_block_constants<" << R << ", " << block
          << ">(bp.kp[" << k << "], s_grid, cpl, mass_r); break;\n";
    o << "      }\n      __syncthreads();\n      cur = k;\n    }\n"
      << "    const long long first = (item - bp.start[k]) * bp.group[k];\n"
      << "    const long long last = first + bp.group[k] < bp.ntiles[k] ? first + bp.group[k] : bp.ntiles[k];\n"
      << "    for (long long tile = first; tile < last; ++tile) {\n"
      << "      switch (k) {\n";
    for (size_t k = 0; k < ps.size(); ++k)
        o << "        case " << k << ": body" << k << "::tile_body<" << R << ", " << block << ", " << hts[k]
          << ">(bp.kp[" << k << "], tile, smem_raw, s_grid, cpl, mass_r); break;\n";
    o << "      }\n    }\n  }\n}\n";
    return o.str();
}

}  // namespace mfi
