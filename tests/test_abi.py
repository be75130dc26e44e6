"""Host-side tests of the C ABI (CPU only: no GPU call is made).

* the shared library loads and exports every function include/madflow_gb.h
  declares, and the Python binding declares the same names;
* descriptor validation rejects malformed programs with MF_EINVAL or
  MF_EUNSUPPORTED (through mf_generate_kernel_source, which validates exactly
  like mf_create_process but needs no device);
* the generated process kernels (integrand and gradient) compile for
  sm_103a with NVRTC.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    from paper_2106_10279_gb300 import _lib
    return _lib


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(mf_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(built):
    lib = C.CDLL(built.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(built.SIGNATURES), set(declared) ^ set(built.SIGNATURES)


def test_struct_layouts_match_the_c_compiler(built, tmp_path):
    # sizes and field offsets of every ABI struct as gcc lays them out from
    # the header, against the ctypes mirror used by the binding
    structs = {"mf_op": built.mf_op, "mf_colour_term": built.mf_colour_term,
               "mf_process_desc": built.mf_process_desc, "mf_process_info": built.mf_process_info,
               "mf_iter_result": built.mf_iter_result, "mf_lhe_init": built.mf_lhe_init,
               "mf_observable": built.mf_observable}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "madflow_gb.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            cname = "in" if fname == "in_" else fname
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {cname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        sname, what, val = line.split()
        cls = structs[sname]
        got = C.sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert got == int(val), line


def _desc(name="gg_ttx"):
    from paper_2106_10279_gb300 import api
    return api.descriptor_for_workload(W.WORKLOADS[name])


def _status(built, d, prec=0, compile_=0):
    n = C.c_size_t(0)
    return built.lib().mf_generate_kernel_source(C.byref(d.desc), prec, compile_, None, C.byref(n))


def test_valid_descriptors_pass_validation(built):
    for name in W.WORKLOADS:
        assert _status(built, _desc(name)) == built.MF_OK, name


@pytest.mark.parametrize("mutate,expect", [
    (lambda d: setattr(d.desc, "n_legs", 2), "MF_EINVAL"),
    (lambda d: setattr(d.desc, "n_legs", 9), "MF_EUNSUPPORTED"),
    (lambda d: setattr(d.desc, "colour_den", 0), "MF_EINVAL"),
    (lambda d: setattr(d.desc, "sqrt_s", -1.0), "MF_EINVAL"),
    (lambda d: setattr(d.desc, "n_couplings", 0), "MF_EINVAL"),
    (lambda d: setattr(d.desc, "average", 0.0), "MF_EINVAL"),
    (lambda d: setattr(d.desc, "pdf_nx", 2), "MF_EINVAL"),
    (lambda d: setattr(d.desc, "mu_f2", 0.0), "MF_EINVAL"),
    (lambda d: setattr(d.desc, "n_jamp", 200), "MF_EUNSUPPORTED"),
])
def test_malformed_descriptors_are_rejected(built, mutate, expect):
    d = _desc()
    mutate(d)
    assert _status(built, d) == getattr(built, expect)
    assert built.lib().mf_last_error()


def test_bad_ops_are_rejected(built):
    d = _desc()
    ops = d.desc.ops
    # an op reading a wavefunction that comes later
    saved = ops[4].in_[0]
    ops[4].in_[0] = 6
    assert _status(built, d) == built.MF_EINVAL
    ops[4].in_[0] = saved
    # a colour term outside the flows
    t = d.desc.terms
    saved = t[0].jamp
    t[0].jamp = 5
    assert _status(built, d) == built.MF_EINVAL
    t[0].jamp = saved
    # asymmetric colour matrix
    d.desc.colour_num[1] += 1
    assert _status(built, d) == built.MF_EINVAL
    d.desc.colour_num[1] -= 1
    assert _status(built, d) == built.MF_OK


def test_null_and_range_arguments(built):
    lib = built.lib()
    assert lib.mf_create_process(None, None) == built.MF_EINVAL
    h = C.c_void_p()
    assert lib.mf_vegas_create(0, 50, 1.5, C.byref(h)) == built.MF_EINVAL
    assert lib.mf_vegas_create(4, 1, 1.5, C.byref(h)) == built.MF_EINVAL
    assert lib.mf_vegas_create(4, 300, 1.5, C.byref(h)) == built.MF_EINVAL
    assert lib.mf_integrand(None, None, 10, None, 0, None) == built.MF_EINVAL
    assert lib.mf_destroy_process(None) == built.MF_OK
    assert lib.mf_vegas_destroy(None) == built.MF_OK


@pytest.mark.parametrize("name", ["ee_mumu", "gg_ttx", "uux_ttx", "gg_ttxg", "uux_ttxg"])
def test_generated_kernels_compile_for_sm103a(built, name):
    from paper_2106_10279_gb300 import api
    d = _desc(name)
    for prec in ("fp64", "mixed"):
        src = api.mf_generate_kernel_source(d, prec, compile=True)
        assert "mf_kernel" in src and "helicity_msq" in src


@pytest.mark.parametrize("name", ["ee_mumu", "gg_ttx", "uux_ttxg"])
def test_gradient_kernels_compile_for_sm103a(built, name):
    from paper_2106_10279_gb300 import api
    src = api.mf_generate_kernel_source(_desc(name), "grad", compile=True)
    assert "mf_grad_kernel" in src and "helicity_grad" in src


def test_batched_kernel_of_the_mixed_batch_compiles(built):
    # the five subprocesses of the mixed batch in one module, costliest first
    from paper_2106_10279_gb300 import api
    names = ["gg_ttxgg", "gg_ttxg", "uux_ttxg", "gg_ttx", "uux_ttx"]
    src = api.mf_generate_batch_source([_desc(n) for n in names], "mixed", compile=True)
    assert "mf_batch_kernel" in src
    for k in range(5):
        assert f"namespace proc{k}" in src and f"body{k}::tile_body" in src
    from paper_2106_10279_gb300 import _lib as L
    with pytest.raises(L.MfError):
        api.mf_generate_batch_source([_desc("gg_ttx")] * 9, "mixed")


def test_measure_peak_rejects_bad_arguments_without_a_device(built):
    # argument checks come before any CUDA call
    lib = built.lib()
    tf = C.c_double()
    assert lib.mf_measure_peak(7, 1, C.byref(tf), None, None) == built.MF_EINVAL
    assert lib.mf_measure_peak(0, 0, C.byref(tf), None, None) == built.MF_EINVAL
    assert lib.mf_measure_peak(0, 1, None, None, None) == built.MF_EINVAL


def test_process_options_reach_the_generator_and_are_checked(built):
    from paper_2106_10279_gb300 import api
    wl = W.WORKLOADS["gg_ttxg"]
    plain = api.mf_generate_kernel_source(api.descriptor_for_workload(wl, options={"amplitude_units": 0}), "fp64")
    units = api.mf_generate_kernel_source(api.descriptor_for_workload(wl), "fp64")
    inline = api.mf_generate_kernel_source(api.descriptor_for_workload(wl, options={"call_routines": 0}), "fp64")
    assert "vs.c[c]" not in plain and "vs.c[c]" in units      # summed vector currents of a unit (the default)
    assert "nFFV_AMP" in plain and "nFFV_AMP" not in inline    # amplitude routines called / inlined
    for bad in ({"amplitude_units": 2}, {"call_routines": 4}, {"block": 192}, {"lanes": 12}, {"ptxas_level": 4},
                {"blocks_per_sm": 0}, {"min_blocks": 9}):
        d = api.descriptor_for_workload(wl, options=bad)
        n = C.c_size_t(0)
        assert built.lib().mf_generate_kernel_source(C.byref(d.desc), 0, 0, None, C.byref(n)) == built.MF_EINVAL, bad
