// Code generation: the diagram program of an mf_process becomes straight-line
// CUDA (one function per helicity evaluation), so that every wavefunction lives
// in registers and every routine is inlined.  This replaces the paper's
// exporter to TensorFlow (Sec. 2.2) with specialisation at run time.
#include <cmath>
#include <cstdio>
#include <map>
#include <sstream>

#include "mf_internal.h"

namespace mfi {
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

}  // namespace

std::string generate_source(const mf_process &p, int precision, int block, int ht, GenInfo &info) {
    const char *R = precision == MF_FP64 ? "double" : "float";
    const int n = p.n_legs;
    std::ostringstream o;
    // --- wavefunction momenta as signed leg masks, denominator slots
    std::vector<uint32_t> mask(p.ops.size(), 0);
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
    o << "namespace proc {\n";
    o << "constexpr int NLEG = " << n << ", NOUT = " << p.n_out << ", NDIM = " << p.ndim
      << ", NJAMP = " << p.n_jamp << ", NDEN = " << info.n_den << ", HADRONIC = " << p.hadronic << ";\n";
    o << "constexpr int LEG_MASS_ID[NLEG] = {";
    for (int i = 0; i < n; ++i) o << (i ? ", " : "") << p.leg_mass_id[i];
    o << "};\n";
    std::vector<int> cuts;
    for (int i = 0; i < n; ++i)
        if (p.leg_cut[i] && !p.leg_incoming[i]) cuts.push_back(i);
    o << "constexpr int NCUT = " << cuts.size() << ";\n";
    o << "constexpr int CUT_LEGS[" << (cuts.empty() ? 1 : cuts.size()) << "] = {";
    if (cuts.empty()) o << "0";
    for (size_t i = 0; i < cuts.size(); ++i) o << (i ? ", " : "") << cuts[i];
    o << "};\n";

    // --- propagator denominators from double-precision invariants
    o << "MF_DEV void denominators(const double (*p)[4], const double *masses, double *den) {\n";
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
                o << "  const double d" << i << "_" << j << " = " << (sg > 0 ? "" : "-")
                  << "2.0 * (p[" << i << "][0] * p[" << j << "][0] - p[" << i << "][1] * p[" << j
                  << "][1] - p[" << i << "][2] * p[" << j << "][2] - p[" << i << "][3] * p[" << j
                  << "][3]);\n";
            }
    for (int s = 0; s < info.n_den; ++s) {
        const DenSlot &d = info.dens[s];
        // P^2 - M^2 = (sum of the legs' m^2 - M^2) + sum of 2 P_i.P_j: the mass
        // terms first, so that an on-shell mass cancels exactly before the
        // (possibly small) invariants are added
        o << "  den[" << s << "] = (0.0";
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

    // --- the program for one helicity
    o << "template <typename R>\n"
         "MF_DEV R helicity_msq(const R (*mom)[4], const R *__restrict__ idn, const int8_t *hel,\n"
         "                      const mf::cx<R> *cpl, const R *mass) {\n"
         "  using namespace mf;\n";
    double fl = 0.0;
    for (size_t k = 0; k < p.ops.size(); ++k) {
        const mf_op &op = p.ops[k];
        fl += routine_flops(op.routine);
        auto M = [&](int id) { return id >= 0 ? "mass[" + std::to_string(id) + "]" : std::string("R(0)"); };
        if (op.kind == MF_OP_EXT) {
            int l = op.leg;
            const char *sg = p.leg_incoming[l] ? "R(1)" : "R(-1)";
            if (op.routine == MF_R_VXX) {
                o << "  const W<R> w" << k << " = vxx<R>(mom[" << l << "], hel[" << l << "], " << sg << ");\n";
            } else {
                // column: u (incoming particle) or v (outgoing antiparticle);
                // row: u-bar (outgoing particle) or v-bar (incoming antiparticle)
                int anti = (op.routine == MF_R_IXX) ? (p.leg_incoming[l] ? 0 : 1) : (p.leg_incoming[l] ? 1 : 0);
                o << "  const W<R> w" << k << " = " << (op.routine == MF_R_IXX ? "ixx" : "oxx") << "<R>(mom[" << l
                  << "], " << M(p.leg_mass_id[l]) << ", hel[" << l << "], " << anti << ", " << sg << ");\n";
            }
        } else if (op.kind == MF_OP_CUR) {
            std::string g = "cpl[" + std::to_string(op.coupling) + "]";
            std::string den = "idn[" + std::to_string(info.op_den[k]) + "]";
            o << "  const W<R> w" << k << " = ";
            switch (op.routine) {
                case MF_R_FFV_FIN: o << "FFV_FIN<R>(w" << op.in[0] << ", w" << op.in[1] << ", " << g << ", " << M(op.mass_id) << ", " << den << ")"; break;
                case MF_R_FFV_FOUT: o << "FFV_FOUT<R>(w" << op.in[0] << ", w" << op.in[1] << ", " << g << ", " << M(op.mass_id) << ", " << den << ")"; break;
                case MF_R_FFV_VEC: o << "FFV_VEC<R>(w" << op.in[0] << ", w" << op.in[1] << ", " << g << ", " << den << ")"; break;
                case MF_R_VVV_VEC: o << "VVV_VEC<R>(w" << op.in[0] << ", w" << op.in[1] << ", " << g << ", " << den << ")"; break;
                case MF_R_VVVV1_VEC: case MF_R_VVVV2_VEC: case MF_R_VVVV3_VEC:
                    o << "VVVV_VEC<R, " << (op.routine - MF_R_VVVV1_VEC + 1) << ">(w" << op.in[0] << ", w" << op.in[1]
                      << ", w" << op.in[2] << ", " << g << ", " << den << ")";
                    break;
                default: o << "/* bad routine */ w0"; break;
            }
            o << ";\n";
        }
    }
    // amplitudes
    o << "  cx<R> J[NJAMP];\n#pragma unroll\n  for (int k = 0; k < NJAMP; ++k) J[k] = C<R>(R(0), R(0));\n";
    for (size_t k = 0; k < p.ops.size(); ++k) {
        const mf_op &op = p.ops[k];
        if (op.kind != MF_OP_AMP) continue;
        std::string g = "cpl[" + std::to_string(op.coupling) + "]";
        o << "  { const cx<R> a = ";
        switch (op.routine) {
            case MF_R_FFV_AMP: o << "FFV_AMP<R>(w" << op.in[0] << ", w" << op.in[1] << ", w" << op.in[2] << ", " << g << ")"; break;
            case MF_R_VVV_AMP: o << "VVV_AMP<R>(w" << op.in[0] << ", w" << op.in[1] << ", w" << op.in[2] << ", " << g << ")"; break;
            default:
                o << "VVVV_AMP<R, " << (op.routine - MF_R_VVVV1_AMP + 1) << ">(w" << op.in[0] << ", w" << op.in[1]
                  << ", w" << op.in[2] << ", w" << op.in[3] << ", " << g << ")";
        }
        o << ";\n";
        for (int t = 0; t < op.n_terms; ++t) {
            const mf_colour_term &ct = p.terms[op.first_term + t];
            std::string Jk = "J[" + std::to_string(ct.jamp) + "]";
            fl += 8;
            if (ct.im == 0.0 && ct.re == 1.0) o << "    " << Jk << " = " << Jk << " + a;\n";
            else if (ct.im == 0.0 && ct.re == -1.0) o << "    " << Jk << " = " << Jk << " - a;\n";
            else if (ct.re == 0.0 && ct.im == 1.0) o << "    " << Jk << " = " << Jk << " + mul_i(a);\n";
            else if (ct.re == 0.0 && ct.im == -1.0) o << "    " << Jk << " = " << Jk << " - mul_i(a);\n";
            else
                o << "    " << Jk << " = cfma(C<R>(R(" << fmt_double(ct.re) << "), R(" << fmt_double(ct.im)
                  << ")), a, " << Jk << ");\n";
        }
        o << "  }\n";
    }
    // colour sum  sum_kl Re(conj(J_k) C_kl J_l) / den, C symmetric:
    // sum_k Re(conj(J_k) (C_kk J_k + 2 sum_{l>k} C_kl J_l))
    o << "  R m = R(0);\n";
    const int nj = p.n_jamp;
    for (int k = 0; k < nj; ++k) {
        o << "  { cx<R> z = R(" << p.colour_num[k * nj + k] << ") * J[" << k << "];\n";
        for (int l = k + 1; l < nj; ++l) {
            int c = p.colour_num[k * nj + l];
            if (c == 0) continue;
            o << "    z = z + R(" << 2 * c << ") * J[" << l << "];\n";
        }
        o << "    m += J[" << k << "].re * z.re + J[" << k << "].im * z.im; }\n";
    }
    fl += 4.0 * nj * (nj - 1) / 2 + 6.0 * nj;
    o << "  return m * R(" << fmt_double(1.0 / p.colour_den) << ");\n}\n";
    o << "}  // namespace proc\n";
    o << "#include \"mf_kernel.cuh\"\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << block << ") mf_kernel(const mf::KParams kp) {\n"
      << "  mf::kernel_body<" << R << ", " << block << ", " << ht << ">(kp);\n}\n";
    info.flops_per_hel = fl;
    // kinematics per event (phase space, PDFs, denominators), rough count
    info.flops_kin = 400.0 + 10.0 * info.n_den;
    return o.str();
}

}  // namespace mfi
