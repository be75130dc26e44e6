"""ctypes declarations of the C ABI in include/madflow_gb.h (argument
marshalling only; every computation happens in libmadflow_gb.so).

Importing this module loads the in-tree library and raises if it is missing:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmadflow_gb.so")

MF_OK, MF_EINVAL, MF_ENOMEM, MF_ECUDA, MF_ENAN, MF_ETIMEOUT, MF_EUNSUPPORTED, MF_EJIT = range(8)
MF_FP64, MF_MIXED, MF_MIXED_TC = 0, 1, 3
STATUS_NAMES = {0: "MF_OK", 1: "MF_EINVAL", 2: "MF_ENOMEM", 3: "MF_ECUDA", 4: "MF_ENAN",
                5: "MF_ETIMEOUT", 6: "MF_EUNSUPPORTED", 7: "MF_EJIT"}

c_i32 = C.c_int32
c_i64 = C.c_int64
P = C.POINTER


class mf_op(C.Structure):
    _fields_ = [("kind", c_i32), ("routine", c_i32), ("in_", c_i32 * 4), ("leg", c_i32),
                ("coupling", c_i32), ("mass_id", c_i32), ("first_term", c_i32), ("n_terms", c_i32)]


class mf_colour_term(C.Structure):
    _fields_ = [("jamp", c_i32), ("pad_", c_i32), ("re", C.c_double), ("im", C.c_double)]


class mf_process_options(C.Structure):
    _fields_ = [("amplitude_units", c_i32), ("call_routines", c_i32), ("order_search", c_i32),
                ("sync_every", c_i32), ("program_parts", c_i32), ("min_blocks", c_i32), ("helicity_pairs", c_i32),
                ("block", c_i32), ("lanes", c_i32), ("blocks_per_sm", c_i32), ("ptxas_level", c_i32),
                ("wait_polls", c_i32)]


MF_OPT_AUTO = -1


class mf_process_desc(C.Structure):
    _fields_ = [
        ("n_legs", c_i32), ("leg_kind", P(c_i32)), ("leg_incoming", P(c_i32)), ("leg_mass_id", P(c_i32)),
        ("leg_cut", P(c_i32)), ("n_masses", c_i32), ("masses", P(C.c_double)),
        ("n_ops", c_i32), ("ops", P(mf_op)), ("n_terms", c_i32), ("terms", P(mf_colour_term)),
        ("n_couplings", c_i32), ("couplings", P(C.c_double)),
        ("n_jamp", c_i32), ("colour_num", P(c_i32)), ("colour_den", c_i32),
        ("n_hel", c_i32), ("helicities", P(C.c_int8)),
        ("average", C.c_double), ("alpha_s_power", c_i32), ("alpha_s", C.c_double),
        ("sqrt_s", C.c_double), ("hadronic", c_i32), ("pdf", P(C.c_double) * 2),
        ("pdf_nx", c_i32), ("pdf_nq", c_i32), ("pdf_x_min", C.c_double), ("pdf_x_max", C.c_double),
        ("pdf_q2_min", C.c_double), ("pdf_q2_max", C.c_double), ("mu_f2", C.c_double),
        ("pt_min", C.c_double), ("dr_min", C.c_double), ("options", P(mf_process_options)),
    ]


class mf_process_info(C.Structure):
    _fields_ = [("ndim", c_i32), ("n_legs", c_i32), ("n_hel", c_i32), ("n_hel_all", c_i32),
                ("n_jamp", c_i32), ("n_ops", c_i32), ("n_den", c_i32),
                ("flops_per_hel", C.c_double), ("flops_kinematics", C.c_double),
                ("pair_leg", c_i32), ("n_pairs", c_i32), ("flops_helicity_sum", C.c_double),
                ("helicity_sampling", c_i32)]


class mf_observable(C.Structure):
    _fields_ = [("kind", c_i32), ("leg", c_i32), ("nbins", c_i32), ("pad", c_i32), ("lo", C.c_double),
                ("hi", C.c_double)]


MF_OBS_PT, MF_OBS_RAPIDITY, MF_OBS_PSEUDORAPIDITY = 0, 1, 2
MF_MAX_OBSERVABLES = 4


class mf_lhe_init(C.Structure):
    _fields_ = [("n_legs", c_i32), ("pdg", c_i32 * 8), ("mass", C.c_double * 8), ("beam_pdg", c_i32 * 2),
                ("beam_energy", C.c_double * 2), ("xsec", C.c_double), ("xsec_error", C.c_double),
                ("w_max", C.c_double), ("process_id", c_i32), ("scale", C.c_double), ("alpha_qed", C.c_double),
                ("alpha_s", C.c_double), ("n_flows", c_i32), ("pad", c_i32), ("colour_tags", P(c_i32))]


class mf_iter_result(C.Structure):
    _fields_ = [("iteration", c_i32), ("n_events", c_i64), ("n_nonzero", c_i64), ("n_nan", c_i64),
                ("integral", C.c_double), ("error", C.c_double), ("sigma", C.c_double),
                ("sigma_error", C.c_double), ("chi2_dof", C.c_double)]


# name -> (restype, argtypes)
SIGNATURES = {
    "mf_create_process": (c_i32, [P(mf_process_desc), P(C.c_void_p)]),
    "mf_destroy_process": (c_i32, [C.c_void_p]),
    "mf_process_get_info": (c_i32, [C.c_void_p, P(mf_process_info)]),
    "mf_integrand": (c_i32, [C.c_void_p, C.c_void_p, c_i64, C.c_void_p, c_i32, C.c_void_p]),
    "mf_helicity_msq": (c_i32, [C.c_void_p, C.c_void_p, c_i64, C.c_void_p, c_i32, C.c_void_p]),
    "mf_grad": (c_i32, [C.c_void_p, C.c_void_p, c_i64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mf_grad_channel": (c_i32, [C.c_void_p, c_i32, C.c_void_p, c_i64, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p]),
    "mf_vegas_create": (c_i32, [c_i32, c_i32, C.c_double, P(C.c_void_p)]),
    "mf_vegas_destroy": (c_i32, [C.c_void_p]),
    "mf_vegas_iterate": (c_i32, [P(C.c_void_p), P(C.c_void_p), P(c_i64), c_i32, C.c_uint64, c_i32, c_i32,
                                 P(mf_iter_result), C.c_void_p]),
    "mf_process_last_kernel_ms": (c_i32, [C.c_void_p, P(C.c_double)]),
    "mf_process_channels": (c_i32, [C.c_void_p, P(c_i32)]),
    "mf_process_set_channel_regulators": (c_i32, [C.c_void_p, C.c_double, C.c_double]),
    "mf_channel_integrand": (c_i32, [C.c_void_p, c_i32, C.c_void_p, c_i64, C.c_void_p, c_i32, C.c_void_p]),
    "mf_vegas_iterate_channels": (c_i32, [P(C.c_void_p), C.c_void_p, P(c_i64), c_i32, C.c_uint64, c_i32, c_i32,
                                          P(mf_iter_result), C.c_void_p]),
    "mf_channels_allocate": (c_i32, [c_i32, P(C.c_double), P(c_i64), C.c_double, c_i64, c_i64, P(c_i64)]),
    "mf_vegas_unweight_channel": (c_i32, [C.c_void_p, C.c_void_p, c_i32, c_i64, C.c_uint64, c_i32, C.c_double,
                                          C.c_void_p, P(C.c_double), c_i64, P(c_i64), C.c_void_p]),
    "mf_process_channel_max_weights": (c_i32, [C.c_void_p, P(c_i64), c_i32, P(C.c_double), C.c_void_p]),
    "mf_channels_describe": (c_i32, [P(mf_process_desc), P(c_i32), P(c_i32), c_i32]),
    "mf_channels_table": (c_i32, [P(mf_process_desc), P(c_i32), P(c_i32)]),
    "mf_vegas_get_grid": (c_i32, [C.c_void_p, P(C.c_double)]),
    "mf_vegas_set_grid": (c_i32, [C.c_void_p, P(C.c_double)]),
    "mf_vegas_get_histogram": (c_i32, [C.c_void_p, P(C.c_double), P(c_i64)]),
    "mf_vegas_get_shape": (c_i32, [C.c_void_p, P(c_i32), P(c_i32), P(c_i32)]),
    "mf_vegas_partial_size": (c_i32, [C.c_void_p, P(c_i32)]),
    "mf_vegas_shard_accumulate": (c_i32, [C.c_void_p, C.c_void_p, c_i64, c_i64, c_i64, c_i32, C.c_uint64, c_i32,
                                          P(C.c_double), P(c_i32), C.c_void_p]),
    "mf_vegas_shard_finish": (c_i32, [C.c_void_p, c_i64, P(C.c_double), c_i32, c_i32, P(mf_iter_result),
                                      C.c_void_p]),
    "mf_tree_frontier": (c_i32, [c_i64, c_i64, c_i64, P(c_i64), c_i32, P(c_i32)]),
    "mf_tree_reduce": (c_i32, [P(C.c_double), c_i32, c_i32, c_i64, c_i32, c_i64, P(C.c_double)]),
    "mf_vegas_iterate_static": (c_i32, [C.c_void_p, C.c_void_p, c_i64, C.c_uint64, c_i32, c_i32,
                                        P(mf_iter_result), C.c_void_p]),
    "mf_process_check": (c_i32, [C.c_void_p]),
    "mf_process_kernel_info": (c_i32, [C.c_void_p, c_i32, P(c_i32), P(c_i32), P(c_i32), P(c_i32), P(c_i32)]),
    "mf_process_set_helicity_sampling": (c_i32, [C.c_void_p, c_i32, C.c_uint64]),
    "mf_process_set_leading_colour": (c_i32, [C.c_void_p, c_i32]),
    "mf_process_set_colour_sampling": (c_i32, [C.c_void_p, c_i32]),
    "mf_process_get_helicities": (c_i32, [C.c_void_p, P(C.c_int8), P(c_i32)]),
    "mf_process_get_helicity_pairs": (c_i32, [C.c_void_p, P(c_i32), P(c_i32)]),
    "mf_process_tune": (c_i32, [C.c_void_p, c_i32, c_i64, C.c_void_p, P(c_i32), P(c_i32)]),
    "mf_batch_create": (c_i32, [P(C.c_void_p), c_i32, c_i32, P(C.c_void_p)]),
    "mf_batch_destroy": (c_i32, [C.c_void_p]),
    "mf_batch_iterate": (c_i32, [C.c_void_p, P(C.c_void_p), P(c_i64), C.c_uint64, c_i32, P(mf_iter_result),
                                 C.c_void_p]),
    "mf_batch_iterate_graph": (c_i32, [C.c_void_p, P(C.c_void_p), P(c_i64), C.c_uint64, c_i32, P(mf_iter_result),
                                       C.c_void_p]),
    "mf_batch_get_info": (c_i32, [C.c_void_p, P(c_i32), P(c_i32), P(C.c_double)]),
    "mf_generate_batch_source": (c_i32, [P(P(mf_process_desc)), c_i32, c_i32, c_i32, C.c_char_p, P(C.c_size_t)]),
    "mf_lhe_open": (c_i32, [C.c_char_p, P(mf_lhe_init), P(C.c_void_p)]),
    "mf_lhe_close": (c_i32, [C.c_void_p, P(c_i64)]),
    "mf_lhe_write": (c_i32, [C.c_void_p, P(C.c_double), c_i64]),
    "mf_vegas_unweight": (c_i32, [C.c_void_p, C.c_void_p, c_i64, C.c_uint64, c_i32, c_i32, C.c_double, C.c_void_p,
                                  P(C.c_double), c_i64, P(c_i64), C.c_void_p]),
    "mf_process_read_weights": (c_i32, [C.c_void_p, P(c_i64), c_i64, P(C.c_double)]),
    "mf_vegas_observables": (c_i32, [C.c_void_p, C.c_void_p, c_i64, C.c_uint64, c_i32, c_i32, c_i32,
                                     P(mf_observable), P(C.c_double), P(C.c_double), P(c_i64), C.c_void_p]),
    "mf_vegas_observables_channel": (c_i32, [C.c_void_p, C.c_void_p, c_i32, c_i64, C.c_uint64, c_i32, c_i32,
                                             P(mf_observable), P(C.c_double), P(C.c_double), P(c_i64),
                                             C.c_void_p]),
    "mf_process_max_weight": (c_i32, [C.c_void_p, P(C.c_double), C.c_void_p]),
    "mf_vegas_save": (c_i32, [C.c_void_p, C.c_void_p, P(C.c_size_t)]),
    "mf_vegas_load": (c_i32, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "mf_generate_kernel_source": (c_i32, [P(mf_process_desc), c_i32, c_i32, C.c_char_p, P(C.c_size_t)]),
    "mf_colour_sum": (c_i32, [C.c_void_p, c_i64, P(c_i32), c_i32, c_i32, c_i32, C.c_void_p, C.c_void_p]),
    "mf_debug_fail_allocation": (c_i32, [c_i64]),
    "mf_process_options_init": (c_i32, [P(mf_process_options)]),
    "mf_measure_peak": (c_i32, [c_i32, c_i32, P(C.c_double), P(C.c_double), C.c_void_p]),
    "mf_last_error": (C.c_char_p, []),
}

MF_CHUNK = 4096
MF_MAX_TREE_NODES = 128
MF_STATIC_MAX_EVENTS = 262144

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no fallback path exists)")
        _lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


class MfError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib().mf_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def check(status, where, allow=(MF_OK,)):
    if status not in allow:
        raise MfError(status, where)
    return status
