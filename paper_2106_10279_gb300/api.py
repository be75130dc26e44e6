"""Python binding of libmadflow_gb: the C entry points under the same names,
plus small convenience classes.  Marshalling only: torch tensors provide device
memory and streams, every computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from .process import ProcessProgram, build_program

MF_FP64, MF_MIXED = L.MF_FP64, L.MF_MIXED
_PREC = {"fp64": L.MF_FP64, "mixed": L.MF_MIXED, "mixed_tc": L.MF_MIXED_TC, L.MF_FP64: L.MF_FP64,
         L.MF_MIXED: L.MF_MIXED, L.MF_MIXED_TC: L.MF_MIXED_TC, "grad": 2}


def _arr(ctype, values):
    values = list(values)
    return (ctype * max(len(values), 1))(*values)


class Descriptor:
    """An mf_process_desc and the host arrays it points into (kept alive)."""

    def __init__(self, prog: ProcessProgram, *, sqrt_s: float, m_top: float, alpha_s: float,
                 pdf_tables=None, pdf_axes=None, mu_f2: float = 0.0, pt_min: float = 0.0,
                 dr_min: float = 0.0, helicities=None, options=None):
        n = len(prog.legs)
        self.prog = prog
        masses = [m_top]
        leg_mass_id = []
        for m in prog.leg_mass:
            if m == 0.0:
                leg_mass_id.append(-1)
            elif abs(m - m_top) < 1e-12 * m_top:
                leg_mass_id.append(0)
            else:
                masses.append(m)
                leg_mass_id.append(len(masses) - 1)
        ops, terms = [], []
        for op in prog.ops:
            o = L.mf_op()
            o.kind, o.routine = op.kind, op.routine
            ins = list(op.inputs) + [-1] * (4 - len(op.inputs))
            for q in range(4):
                o.in_[q] = ins[q]
            o.leg = op.leg
            o.coupling = op.coupling
            if op.kind == 1 and op.mass != 0.0:
                o.mass_id = 0 if abs(op.mass - m_top) < 1e-12 * m_top else masses.index(op.mass)
            else:
                o.mass_id = -1
            o.first_term = len(terms)
            o.n_terms = len(op.terms)
            for (k, re, im) in op.terms:
                terms.append(L.mf_colour_term(k, 0, re, im))
            ops.append(o)
        cut = [0] * n
        if pt_min > 0 or dr_min > 0:
            for i, (p, inc) in enumerate(prog.legs):
                if p == "g" and not inc:
                    cut[i] = 1
        self._keep = []
        d = L.mf_process_desc()
        d.n_legs = n
        d.leg_kind = self._k(_arr(C.c_int32, prog.leg_kind))
        d.leg_incoming = self._k(_arr(C.c_int32, [1 if inc else 0 for _, inc in prog.legs]))
        d.leg_mass_id = self._k(_arr(C.c_int32, leg_mass_id))
        d.leg_cut = self._k(_arr(C.c_int32, cut))
        d.n_masses = len(masses)
        d.masses = self._k(_arr(C.c_double, masses))
        d.n_ops = len(ops)
        d.ops = self._k((L.mf_op * len(ops))(*ops))
        d.n_terms = len(terms)
        d.terms = self._k((L.mf_colour_term * max(len(terms), 1))(*terms))
        cpl = []
        for c in prog.couplings:
            cpl += [float(np.real(c)), float(np.imag(c))]
        d.n_couplings = len(prog.couplings)
        d.couplings = self._k(_arr(C.c_double, cpl))
        nj = prog.colour_num.shape[0]
        d.n_jamp = nj
        d.colour_num = self._k(_arr(C.c_int32, [int(v) for v in prog.colour_num.reshape(-1)]))
        d.colour_den = int(prog.colour_den)
        if helicities is not None:
            h = np.asarray(helicities, dtype=np.int8).reshape(-1, n)
            d.n_hel = h.shape[0]
            d.helicities = self._k(_arr(C.c_int8, h.reshape(-1).tolist()))
        d.average = prog.average
        d.alpha_s_power = prog.alpha_s_power
        d.alpha_s = alpha_s
        d.sqrt_s = sqrt_s
        if pdf_tables is not None:
            d.hadronic = 1
            for b in range(2):
                t = np.ascontiguousarray(pdf_tables[b], dtype=np.float64)
                self._keep.append(t)
                d.pdf[b] = t.ctypes.data_as(C.POINTER(C.c_double))
            nq, nx = np.asarray(pdf_tables[0]).shape
            d.pdf_nx, d.pdf_nq = nx, nq
            d.pdf_x_min, d.pdf_x_max, d.pdf_q2_min, d.pdf_q2_max = pdf_axes
            d.mu_f2 = mu_f2
        d.pt_min = pt_min
        d.dr_min = dr_min
        if options:
            o = L.mf_process_options()
            L.check(L.lib().mf_process_options_init(C.byref(o)), "mf_process_options_init")
            for k, v in options.items():
                setattr(o, k, int(v))
            self._keep.append(o)
            d.options = C.pointer(o)
        self.desc = d

    def _k(self, arr):
        self._keep.append(arr)
        return C.cast(arr, C.POINTER(arr._type_))


def descriptor_for_workload(wl, m_top=None, alpha_s=None, q2_slope: float = 0.0, helicities=None, options=None):
    """Descriptor of one of the synthetic workloads (``workloads`` module);
    options: a dict of mf_process_options fields (the rest MF_OPT_AUTO)."""
    import workloads as W
    mt = wl.m_top if m_top is None else m_top
    a_s = wl.alpha_s if alpha_s is None else alpha_s
    prog = build_program(wl.name, [(l.particle, l.incoming) for l in wl.legs], {"t": mt}, a_s, wl.alpha)
    tables = axes = None
    if wl.beams:
        tables = [W.pdf_table(b, q2_slope) for b in wl.beams]
        axes = (W.PDF_X_MIN, W.PDF_X_MAX, W.PDF_Q2_MIN, W.PDF_Q2_MAX)
    return Descriptor(prog, sqrt_s=wl.sqrt_s, m_top=mt, alpha_s=a_s, pdf_tables=tables, pdf_axes=axes,
                      mu_f2=wl.mu_f2, pt_min=wl.pt_min_gluon, dr_min=wl.dr_min_gluon, helicities=helicities,
                      options=options)


# ---------------------------------------------------------------- C entry points
def mf_create_process(desc: Descriptor):
    h = C.c_void_p()
    L.check(L.lib().mf_create_process(C.byref(desc.desc), C.byref(h)), "mf_create_process")
    return h


def mf_destroy_process(h):
    L.check(L.lib().mf_destroy_process(h), "mf_destroy_process")


def mf_process_get_info(h) -> dict:
    info = L.mf_process_info()
    L.check(L.lib().mf_process_get_info(h, C.byref(info)), "mf_process_get_info")
    return {k: getattr(info, k) for k, _ in info._fields_}


def mf_process_last_kernel_ms(h) -> float:
    ms = C.c_double()
    L.check(L.lib().mf_process_last_kernel_ms(h, C.byref(ms)), "mf_process_last_kernel_ms")
    return ms.value


PEAK_KINDS = {"fp32_ffma": 0, "fp64_dfma": 1, "tf32_mma": 2, "fp32_ffma2": 3}


def mf_measure_peak(kind: str, reps: int = 10, stream=None):
    """The device's measured arithmetic peak of one kind (fp32_ffma,
    fp32_ffma2, fp64_dfma or tf32_mma): (TFLOP/s of the best of reps timed launches,
    that launch's ms)."""
    tf, ms = C.c_double(), C.c_double()
    L.check(L.lib().mf_measure_peak(PEAK_KINDS[kind], reps, C.byref(tf), C.byref(ms), _stream_ptr(stream)),
            "mf_measure_peak")
    return tf.value, ms.value


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def mf_integrand(h, x, n: int, f, precision="fp64", stream=None):
    """x, f: device pointers (int) or CUDA tensors (x [ndim, n] float64, f [n] float64)."""
    xp = x if isinstance(x, int) else x.data_ptr()
    fp = f if isinstance(f, int) else f.data_ptr()
    return L.check(L.lib().mf_integrand(h, C.c_void_p(xp), n, C.c_void_p(fp), _PREC[precision],
                                        _stream_ptr(stream)), "mf_integrand")


def mf_helicity_msq(h, x, n: int, out, precision="fp64", stream=None):
    """x [ndim, n] and out [n_hel_all, n] device tensors (or pointers)."""
    xp = x if isinstance(x, int) else x.data_ptr()
    op = out if isinstance(out, int) else out.data_ptr()
    return L.check(L.lib().mf_helicity_msq(h, C.c_void_p(xp), n, C.c_void_p(op), _PREC[precision],
                                           _stream_ptr(stream)), "mf_helicity_msq")


def mf_grad(h, x, n: int, f, df_dparam, df_dx=None, stream=None, channel=None):
    """Device tensors or pointers: x [ndim, n], f [n], df_dparam [2, n], df_dx [ndim, n] or None
    (with a channel: mf_grad_channel)."""
    ptr = lambda t: 0 if t is None else (t if isinstance(t, int) else t.data_ptr())
    if channel is not None:
        return L.check(L.lib().mf_grad_channel(h, channel, C.c_void_p(ptr(x)), n, C.c_void_p(ptr(f)),
                                               C.c_void_p(ptr(df_dparam)), C.c_void_p(ptr(df_dx) or None),
                                               _stream_ptr(stream)), "mf_grad_channel")
    return L.check(L.lib().mf_grad(h, C.c_void_p(ptr(x)), n, C.c_void_p(ptr(f)), C.c_void_p(ptr(df_dparam)),
                                   C.c_void_p(ptr(df_dx) or None), _stream_ptr(stream)), "mf_grad")


def mf_vegas_create(ndim: int, nbins: int = 50, alpha: float = 1.5):
    h = C.c_void_p()
    L.check(L.lib().mf_vegas_create(ndim, nbins, alpha, C.byref(h)), "mf_vegas_create")
    return h


def mf_vegas_destroy(h):
    L.check(L.lib().mf_vegas_destroy(h), "mf_vegas_destroy")


def mf_vegas_iterate(grids, procs, n_events, seed: int, precision="fp64", refine: bool = True, stream=None):
    k = len(grids)
    G = (C.c_void_p * k)(*[g.value for g in grids])
    Pp = (C.c_void_p * k)(*[p.value for p in procs])
    N = (C.c_int64 * k)(*n_events)
    out = (L.mf_iter_result * k)()
    st = L.lib().mf_vegas_iterate(G, Pp, N, k, seed, _PREC[precision], 1 if refine else 0, out,
                                  _stream_ptr(stream))
    L.check(st, "mf_vegas_iterate", allow=(L.MF_OK, L.MF_ENAN))
    return [_result(r) for r in out]


def mf_process_channels(h) -> int:
    n = C.c_int32()
    L.check(L.lib().mf_process_channels(h, C.byref(n)), "mf_process_channels")
    return n.value


def mf_process_set_channel_regulators(h, s0: float, t0: float):
    L.check(L.lib().mf_process_set_channel_regulators(h, float(s0), float(t0)), "mf_process_set_channel_regulators")


def mf_channel_integrand(h, channel: int, x, n: int, f, precision="fp64", stream=None):
    """x [ndim, n], f [n]: device tensors or pointers."""
    xp = x if isinstance(x, int) else x.data_ptr()
    fp = f if isinstance(f, int) else f.data_ptr()
    return L.check(L.lib().mf_channel_integrand(h, channel, C.c_void_p(xp), n, C.c_void_p(fp), _PREC[precision],
                                                _stream_ptr(stream)), "mf_channel_integrand")


def mf_vegas_iterate_channels(grids, h, n_events, seed: int, precision="fp64", refine: bool = True, stream=None):
    k = len(grids)
    G = (C.c_void_p * k)(*[g.value for g in grids])
    N = (C.c_int64 * k)(*[int(v) for v in n_events])
    out = (L.mf_iter_result * k)()
    st = L.lib().mf_vegas_iterate_channels(G, h, N, k, seed, _PREC[precision], 1 if refine else 0, out,
                                           _stream_ptr(stream))
    L.check(st, "mf_vegas_iterate_channels", allow=(L.MF_OK, L.MF_ENAN))
    return [_result(r) for r in out]


def mf_channels_allocate(sigma, n_total: int, n_floor: int, n_prev=None, m0: float = 0.0):
    k = len(sigma)
    S = (C.c_double * k)(*[float(v) for v in sigma])
    Np = None if n_prev is None else (C.c_int64 * k)(*[int(v) for v in n_prev])
    out = (C.c_int64 * k)()
    L.check(L.lib().mf_channels_allocate(k, S, Np, float(m0), int(n_total), int(n_floor), out),
            "mf_channels_allocate")
    return [int(v) for v in out]


def mf_channels_describe(desc: Descriptor):
    """The channel keys of a descriptor's program (host only), in channel order."""
    n = C.c_int32()
    L.check(L.lib().mf_channels_describe(C.byref(desc.desc), C.byref(n), None, 0), "mf_channels_describe")
    stride = 32
    keys = (C.c_int32 * (max(n.value, 1) * stride))()
    L.check(L.lib().mf_channels_describe(C.byref(desc.desc), C.byref(n), keys, stride), "mf_channels_describe")
    out = []
    for i in range(n.value):
        ln = keys[i * stride]
        out.append(tuple(keys[i * stride + 1: i * stride + 1 + ln]))
    return out


def mf_channels_table(desc: Descriptor):
    """The int32 channel table the kernels read (host only)."""
    import numpy as np
    n = C.c_int32(0)
    L.check(L.lib().mf_channels_table(C.byref(desc.desc), None, C.byref(n)), "mf_channels_table")
    buf = (C.c_int32 * max(n.value, 1))()
    L.check(L.lib().mf_channels_table(C.byref(desc.desc), buf, C.byref(n)), "mf_channels_table")
    return np.array(buf[:n.value], dtype=np.int32)


def _result(r):
    return {name: getattr(r, name) for name, _ in r._fields_}


def mf_vegas_partial_size(h) -> int:
    k = C.c_int32()
    L.check(L.lib().mf_vegas_partial_size(h, C.byref(k)), "mf_vegas_partial_size")
    return k.value


def mf_vegas_shard_accumulate(h, proc_h, n_total: int, chunk_begin: int, chunk_end: int, subprocess: int,
                              seed: int, precision="fp64", stream=None):
    """This rank's tree nodes, float64 [n_nodes, 2 + K] (level, index, values)."""
    K = mf_vegas_partial_size(h)
    buf = np.zeros((L.MF_MAX_TREE_NODES, 2 + K))
    nn = C.c_int32()
    st = L.lib().mf_vegas_shard_accumulate(h, proc_h, n_total, chunk_begin, chunk_end, subprocess, seed,
                                           _PREC[precision], buf.ctypes.data_as(C.POINTER(C.c_double)),
                                           C.byref(nn), _stream_ptr(stream))
    L.check(st, "mf_vegas_shard_accumulate")
    return buf[:nn.value].copy()


def mf_vegas_shard_finish(h, n_total: int, nodes, refine: bool = True, stream=None):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, mf_vegas_partial_size(h) + 2)
    out = L.mf_iter_result()
    st = L.lib().mf_vegas_shard_finish(h, n_total, nodes.ctypes.data_as(C.POINTER(C.c_double)), nodes.shape[0],
                                       1 if refine else 0, C.byref(out), _stream_ptr(stream))
    L.check(st, "mf_vegas_shard_finish", allow=(L.MF_OK, L.MF_ENAN))
    return _result(out)


def mf_tree_frontier(chunk_begin: int, chunk_end: int, nchunks: int):
    """(level, index) pairs, int64 [n, 2], of the maximal aligned nodes of a chunk range."""
    ids = np.zeros((L.MF_MAX_TREE_NODES, 2), dtype=np.int64)
    n = C.c_int32()
    L.check(L.lib().mf_tree_frontier(chunk_begin, chunk_end, nchunks, ids.ctypes.data_as(C.POINTER(C.c_int64)),
                                     L.MF_MAX_TREE_NODES, C.byref(n)), "mf_tree_frontier")
    return ids[:n.value].copy()


def mf_tree_reduce(nodes, nchunks: int, level: int, index: int):
    """Values [K] of node (level, index) from records [n, 2 + K] that partition it."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    if nodes.ndim != 2 or nodes.shape[1] < 3:
        raise ValueError("nodes must be [n, 2 + K]")
    K = nodes.shape[1] - 2
    out = np.zeros(K)
    L.check(L.lib().mf_tree_reduce(nodes.ctypes.data_as(C.POINTER(C.c_double)), nodes.shape[0], K, nchunks,
                                   level, index, out.ctypes.data_as(C.POINTER(C.c_double))), "mf_tree_reduce")
    return out


def tree_levels(nchunks: int) -> int:
    L_ = 0
    while (1 << L_) < nchunks:
        L_ += 1
    return L_


def shard_chunks(n_total: int, rank: int, world: int):
    """Chunk range [c0, c1) of rank `rank` out of `world` (whole chunks, balanced)."""
    nchunks = (n_total + L.MF_CHUNK - 1) // L.MF_CHUNK
    return nchunks * rank // world, nchunks * (rank + 1) // world


def pack_nodes(nodes, K: int):
    """Fixed-size float64 record [1 + MF_MAX_TREE_NODES (2 + K)] of one rank's
    tree nodes (count first), for an all-gather of equal-sized buffers."""
    nodes = np.asarray(nodes, dtype=np.float64).reshape(-1, 2 + K)
    if nodes.shape[0] > L.MF_MAX_TREE_NODES:
        raise ValueError("too many tree nodes")
    buf = np.zeros(1 + L.MF_MAX_TREE_NODES * (2 + K))
    buf[0] = nodes.shape[0]
    buf[1:1 + nodes.size] = nodes.ravel()
    return buf


def unpack_nodes(gathered, K: int):
    """All ranks' nodes [n, 2 + K] from the gathered records [world, len]."""
    g = np.asarray(gathered, dtype=np.float64)
    rec = 2 + K
    return np.concatenate([g[r, 1:1 + int(g[r, 0]) * rec].reshape(-1, rec) for r in range(g.shape[0])])


def mf_vegas_save(h) -> bytes:
    n = C.c_size_t(0)
    L.check(L.lib().mf_vegas_save(h, None, C.byref(n)), "mf_vegas_save")
    buf = C.create_string_buffer(n.value)
    L.check(L.lib().mf_vegas_save(h, buf, C.byref(n)), "mf_vegas_save")
    return buf.raw[:n.value]


def mf_vegas_load(h, data: bytes):
    buf = C.create_string_buffer(bytes(data), len(data))
    L.check(L.lib().mf_vegas_load(h, buf, len(data)), "mf_vegas_load")


def mf_vegas_get_grid(h):
    nd, nb, it = C.c_int32(), C.c_int32(), C.c_int32()
    L.check(L.lib().mf_vegas_get_shape(h, C.byref(nd), C.byref(nb), C.byref(it)), "mf_vegas_get_shape")
    g = np.zeros((nd.value, nb.value + 1))
    L.check(L.lib().mf_vegas_get_grid(h, g.ctypes.data_as(C.POINTER(C.c_double))), "mf_vegas_get_grid")
    return g


def mf_vegas_set_grid(h, edges):
    e = np.ascontiguousarray(edges, dtype=np.float64)
    L.check(L.lib().mf_vegas_set_grid(h, e.ctypes.data_as(C.POINTER(C.c_double))), "mf_vegas_set_grid")


def mf_vegas_get_histogram(h):
    nd, nb, it = C.c_int32(), C.c_int32(), C.c_int32()
    L.check(L.lib().mf_vegas_get_shape(h, C.byref(nd), C.byref(nb), C.byref(it)), "mf_vegas_get_shape")
    s = np.zeros((nd.value, nb.value))
    c = np.zeros((nd.value, nb.value), dtype=np.int64)
    L.check(L.lib().mf_vegas_get_histogram(h, s.ctypes.data_as(C.POINTER(C.c_double)),
                                           c.ctypes.data_as(C.POINTER(C.c_int64))), "mf_vegas_get_histogram")
    return s, c


def mf_generate_kernel_source(desc: Descriptor, precision="fp64", compile: bool = False) -> str:
    n = C.c_size_t(0)
    L.check(L.lib().mf_generate_kernel_source(C.byref(desc.desc), _PREC[precision], 0, None, C.byref(n)),
            "mf_generate_kernel_source")
    buf = C.create_string_buffer(n.value)
    L.check(L.lib().mf_generate_kernel_source(C.byref(desc.desc), _PREC[precision], 1 if compile else 0, buf,
                                              C.byref(n)), "mf_generate_kernel_source")
    return buf.value.decode()


def mf_generate_batch_source(descs, precision="mixed", compile: bool = False) -> str:
    k = len(descs)
    arr = (C.POINTER(L.mf_process_desc) * k)(*[C.pointer(d.desc) for d in descs])
    n = C.c_size_t(0)
    L.check(L.lib().mf_generate_batch_source(arr, k, _PREC[precision], 0, None, C.byref(n)),
            "mf_generate_batch_source")
    buf = C.create_string_buffer(n.value)
    L.check(L.lib().mf_generate_batch_source(arr, k, _PREC[precision], 1 if compile else 0, buf, C.byref(n)),
            "mf_generate_batch_source")
    return buf.value.decode()


# ---------------------------------------------------------------- classes
class Process:
    """A compiled process; ``integrand(x)`` evaluates f at points x [ndim, n]."""

    def __init__(self, desc: Descriptor):
        self.desc = desc
        self.handle = mf_create_process(desc)

    @property
    def info(self):
        """Counts of the process (FLOPs as of the kernel compiled last)."""
        return mf_process_get_info(self.handle)

    @property
    def n_diagrams(self):
        """Feynman diagrams of the process's program."""
        return self.desc.prog.n_diagrams

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(descriptor_for_workload(wl, **kw))

    @property
    def ndim(self):
        return self.info["ndim"]

    def integrand(self, x, precision="fp64", out=None, stream=None):
        import torch
        if x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous float64 CUDA tensor [ndim, n]")
        if x.shape[0] != self.ndim:
            raise ValueError(f"x must have {self.ndim} rows")
        n = x.shape[1]
        f = torch.empty(n, dtype=torch.float64, device=x.device) if out is None else out
        mf_integrand(self.handle, x, n, f, precision, stream)
        return f

    @property
    def n_channels(self):
        """Channels of the multichannel phase space (0: the process has none)."""
        return mf_process_channels(self.handle)

    def set_channel_regulators(self, s0: float, t0: float):
        mf_process_set_channel_regulators(self.handle, s0, t0)

    def channel_integrand(self, x, channel: int, precision="fp64", out=None, stream=None):
        """f at points x [ndim, n] through phase-space channel `channel`
        (weight a_i / g_i in place of the flat phase space's)."""
        import torch
        if x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous float64 CUDA tensor [ndim, n]")
        if x.shape[0] != self.ndim:
            raise ValueError(f"x must have {self.ndim} rows")
        n = x.shape[1]
        f = torch.empty(n, dtype=torch.float64, device=x.device) if out is None else out
        mf_channel_integrand(self.handle, channel, x, n, f, precision, stream)
        return f

    def set_colour_sampling(self, on=True):
        """One uniformly drawn colour flow per point instead of the colour
        sum (unbiased; see mf_process_set_colour_sampling)."""
        L.check(L.lib().mf_process_set_colour_sampling(self.handle, 1 if on else 0),
                "mf_process_set_colour_sampling")

    def set_helicity_sampling(self, on=True, seed=0):
        """One uniformly drawn helicity (on=True or 1) or helicity pair (on=2)
        per point instead of the sum (unbiased)."""
        mode = (1 if on else 0) if isinstance(on, bool) else int(on)
        L.check(L.lib().mf_process_set_helicity_sampling(self.handle, mode, seed),
                "mf_process_set_helicity_sampling")

    def set_leading_colour(self, on=True):
        """Keep only the diagonal of the colour matrix (leading colour)."""
        L.check(L.lib().mf_process_set_leading_colour(self.handle, 1 if on else 0), "mf_process_set_leading_colour")

    def helicities(self):
        """The non-vanishing helicity assignments, int8 [n_hel, n_legs]."""
        n = C.c_int32()
        L.check(L.lib().mf_process_get_helicities(self.handle, None, C.byref(n)), "mf_process_get_helicities")
        out = np.zeros((n.value, self.info["n_legs"]), dtype=np.int8)
        L.check(L.lib().mf_process_get_helicities(self.handle, out.ctypes.data_as(C.POINTER(C.c_int8)),
                                                  C.byref(n)), "mf_process_get_helicities")
        return out

    def helicity_pairs(self):
        """Rows of helicities() forming each helicity pair, int32 [n_pairs, 2]
        (pair leg at -1, at +1; -1 where that assignment vanishes)."""
        n = C.c_int32()
        L.check(L.lib().mf_process_get_helicity_pairs(self.handle, None, C.byref(n)), "mf_process_get_helicity_pairs")
        out = np.zeros((n.value, 2), dtype=np.int32)
        L.check(L.lib().mf_process_get_helicity_pairs(self.handle, out.ctypes.data_as(C.POINTER(C.c_int32)),
                                                      C.byref(n)), "mf_process_get_helicity_pairs")
        return out

    def kernel_info(self, precision="mixed"):
        """Launch shape of a compiled kernel: block, lanes per point, registers, blocks per SM."""
        v = [C.c_int32() for _ in range(5)]
        L.check(L.lib().mf_process_kernel_info(self.handle, _PREC[precision], *[C.byref(x) for x in v]),
                "mf_process_kernel_info")
        return dict(zip(("block", "ht", "regs", "blocks_per_sm", "min_blocks"), (x.value for x in v)))

    def check(self):
        """Raise if a bounded wait of one of this process's kernels expired."""
        L.check(L.lib().mf_process_check(self.handle), "mf_process_check")

    def tune(self, precision="mixed", n_sample=200_000, stream=None):
        """Pick the fastest launch shape (same results); returns (block, lanes per event)."""
        b, h = C.c_int32(), C.c_int32()
        L.check(L.lib().mf_process_tune(self.handle, _PREC[precision], n_sample, _stream_ptr(stream), C.byref(b),
                                        C.byref(h)), "mf_process_tune")
        return b.value, h.value

    def grad(self, x, with_dx=True, stream=None, channel=None):
        """(f [n], df/dparam [2, n] (m_t, alpha_s), df/dx [ndim, n] or None);
        with a channel, through that phase-space channel."""
        import torch
        n = x.shape[1]
        f = torch.empty(n, dtype=torch.float64, device=x.device)
        dp = torch.empty((2, n), dtype=torch.float64, device=x.device)
        dx = torch.empty((self.ndim, n), dtype=torch.float64, device=x.device) if with_dx else None
        mf_grad(self.handle, x, n, f, dp, dx, stream, channel)
        return f, dp, dx

    def helicity_msq(self, x, precision="fp64", stream=None):
        """Colour-summed |M|^2 of every helicity row (unaveraged), [n_hel_all, n]."""
        import torch
        n = x.shape[1]
        out = torch.zeros((self.info["n_hel_all"], n), dtype=torch.float64, device=x.device)
        mf_helicity_msq(self.handle, x, n, out, precision, stream)
        return out

    def close(self):
        if self.handle:
            mf_destroy_process(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Vegas:
    def __init__(self, ndim: int, nbins: int = 50, alpha: float = 1.5):
        self.handle = mf_vegas_create(ndim, nbins, alpha)

    def iterate(self, proc: Process, n_events: int, seed: int, precision="fp64", refine=True, stream=None):
        return mf_vegas_iterate([self.handle], [proc.handle], [n_events], seed, precision, refine, stream)[0]

    @property
    def grid(self):
        return mf_vegas_get_grid(self.handle)

    @grid.setter
    def grid(self, edges):
        mf_vegas_set_grid(self.handle, edges)

    def histogram(self):
        return mf_vegas_get_histogram(self.handle)

    def iterate_shard(self, proc: Process, n_total: int, chunk_begin: int, chunk_end: int, seed: int,
                      subprocess: int = 0, precision="fp64", stream=None):
        """This rank's tree nodes of the next iteration (see mf_vegas_shard_accumulate)."""
        return mf_vegas_shard_accumulate(self.handle, proc.handle, n_total, chunk_begin, chunk_end, subprocess,
                                         seed, precision, stream)

    def finish_shards(self, n_total: int, nodes, refine=True, stream=None):
        """Combine every rank's nodes and finish the iteration (see mf_vegas_shard_finish)."""
        return mf_vegas_shard_finish(self.handle, n_total, nodes, refine, stream)

    def save(self) -> bytes:
        return mf_vegas_save(self.handle)

    def load(self, data: bytes):
        mf_vegas_load(self.handle, data)

    def close(self):
        if self.handle:
            mf_vegas_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiChannel:
    """Vegas over the multichannel phase space of a process: one grid per
    channel, the cross section the sum of the channels' integrals, and the
    points of each iteration shared out by Neyman's rule from the previous
    iteration's per-point standard deviations (equal shares first; with
    m0 > 0 each deviation is first shrunk towards the pooled one with m0
    pseudo-points)."""

    def __init__(self, proc: "Process", nbins: int = 50, alpha: float = 1.5, m0: float = 0.0):
        self.proc = proc
        self.K = proc.n_channels
        if self.K == 0:
            raise ValueError("the process has no phase-space channels")
        self.grids = [Vegas(proc.ndim, nbins, alpha) for _ in range(self.K)]
        self.sigma = None
        self.n_prev = None
        self.m0 = m0

    def allocation(self, n_total: int, n_floor=None):
        if n_floor is None:
            n_floor = max(2, n_total // (10 * self.K))
        if self.sigma is None:
            return mf_channels_allocate([0.0] * self.K, n_total, n_floor)
        return mf_channels_allocate(self.sigma, n_total, n_floor, self.n_prev, self.m0)

    def iterate(self, n_total: int, seed: int, precision="fp64", refine=True, adapt=True, n_floor=None,
                stream=None):
        import math
        n = self.allocation(n_total, n_floor)
        res = mf_vegas_iterate_channels([g.handle for g in self.grids], self.proc.handle, n, seed, precision,
                                        refine, stream)
        if adapt:
            self.sigma = [r["error"] * math.sqrt(k) for r, k in zip(res, n)]
            self.n_prev = list(n)
        tot = {
            "n_events": sum(n),
            "integral": sum(r["integral"] for r in res),
            "error": math.sqrt(sum(r["error"] ** 2 for r in res)),
            "sigma": sum(r["sigma"] for r in res),
            "sigma_error": math.sqrt(sum(r["sigma_error"] ** 2 for r in res)),
            "n_nonzero": sum(r["n_nonzero"] for r in res),
            "n_nan": sum(r["n_nan"] for r in res),
            "per_channel": res,
            "allocation": n,
        }
        return tot

    def unweight(self, n_total: int, seed: int, W_max: float, precision="mixed", lhe: LheWriter = None,
                 n_floor=None, stream=None):
        """Unweighted events of one pass of n_total points over the channels
        (the current allocation) against one maximum W_max of the combined
        weights W = w N / n_k: channel k is unweighted against W_max n_k / N,
        so every event weighs W_max / N.  Returns (number kept, records)."""
        n = self.allocation(n_total, n_floor)
        N = sum(n)
        tot, recs = 0, []
        for k, nk in enumerate(n):
            acc, rec = unweight_channel(self.grids[k], self.proc, k, nk, seed, W_max * nk / N, precision, lhe,
                                        stream=stream)
            tot += acc
            recs.append(rec)
        return tot, np.concatenate(recs) if recs else np.zeros((0, 0))

    def observables(self, n_total: int, seed: int, obs, precision="mixed", n_floor=None, stream=None):
        """Weighted histograms of one pass of n_total points over the channels
        (the current allocation): per observable (sigma, error, counts), the
        sums over the channels (errors in quadrature)."""
        n = self.allocation(n_total, n_floor)
        tot = None
        for k, nk in enumerate(n):
            h = observables(self.grids[k], self.proc, nk, seed, obs, precision, stream=stream, channel=k)
            if tot is None:
                tot = [[s.copy(), e ** 2, c.copy()] for s, e, c in h]
            else:
                for t, (s_, e_, c_) in zip(tot, h):
                    t[0] += s_
                    t[1] += e_ ** 2
                    t[2] += c_
        return [(s_, np.sqrt(v_), c_) for s_, v_, c_ in tot]

    def save(self) -> bytes:
        """Checkpoint of every channel's grid and the allocation state."""
        import struct
        parts = [b"MFMC1", struct.pack("<ii", self.K, 0 if self.sigma is None else 1)]
        if self.sigma is not None:
            parts.append(struct.pack("<%dd" % self.K, *self.sigma))
            parts.append(struct.pack("<%dq" % self.K, *self.n_prev))
        for g in self.grids:
            blob = g.save()
            parts.append(struct.pack("<q", len(blob)))
            parts.append(blob)
        return b"".join(parts)

    def load(self, data: bytes):
        import struct
        if data[:5] != b"MFMC1":
            raise ValueError("not a multichannel checkpoint")
        K, has = struct.unpack_from("<ii", data, 5)
        if K != self.K:
            raise ValueError(f"checkpoint of {K} channels, process has {self.K}")
        o = 13
        self.sigma = None
        self.n_prev = None
        if has:
            self.sigma = list(struct.unpack_from("<%dd" % K, data, o))
            o += 8 * K
            self.n_prev = list(struct.unpack_from("<%dq" % K, data, o))
            o += 8 * K
        for g in self.grids:
            (ln,) = struct.unpack_from("<q", data, o)
            o += 8
            g.load(data[o:o + ln])
            o += ln
        if o != len(data):
            raise ValueError("trailing bytes in the checkpoint")

    def close(self):
        for g in self.grids:
            g.close()
        self.grids = []


class LheWriter:
    """An LHE 3.0 file written by a background thread (see mf_lhe_open)."""

    def __init__(self, path, pdg, masses, beam_pdg=(2212, 2212), beam_energy=(6500.0, 6500.0), xsec=0.0,
                 xsec_error=0.0, w_max=0.0, process_id=1, scale=173.0, alpha_qed=1 / 128, alpha_s=0.118,
                 colour_tags=None):
        """colour_tags: [n_flows, n_legs, 2] LHE colour/anticolour tags per
        colour flow (process.lhe_colour_tags), or None (tags 0)."""
        init = L.mf_lhe_init()
        init.n_legs = len(pdg)
        for i, (p, m) in enumerate(zip(pdg, masses)):
            init.pdg[i] = p
            init.mass[i] = m
        init.beam_pdg[:] = list(beam_pdg)
        init.beam_energy[:] = list(beam_energy)
        init.xsec, init.xsec_error, init.w_max = xsec, xsec_error, w_max
        init.process_id, init.scale, init.alpha_qed, init.alpha_s = process_id, scale, alpha_qed, alpha_s
        if colour_tags is not None:
            t = np.ascontiguousarray(colour_tags, dtype=np.int32).reshape(-1, len(pdg), 2)
            init.n_flows = t.shape[0]
            init.colour_tags = t.ctypes.data_as(C.POINTER(C.c_int32))
        h = C.c_void_p()
        L.check(L.lib().mf_lhe_open(str(path).encode(), C.byref(init), C.byref(h)), "mf_lhe_open")
        self.handle = h
        self.n_legs = len(pdg)

    def write(self, records):
        r = np.ascontiguousarray(records, dtype=np.float64).reshape(-1, 4 + 4 * self.n_legs)
        L.check(L.lib().mf_lhe_write(self.handle, r.ctypes.data_as(C.POINTER(C.c_double)), r.shape[0]),
                "mf_lhe_write")

    def close(self) -> int:
        n = C.c_int64(0)
        if self.handle:
            h, self.handle = self.handle, None
            L.check(L.lib().mf_lhe_close(h, C.byref(n)), "mf_lhe_close")
        return n.value

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unweight(grid: "Vegas", proc: "Process", n_events: int, seed: int, w_max: float, precision="mixed",
             subprocess=0, lhe: LheWriter = None, capacity=None, stream=None):
    """Hit-or-miss unweighted events of one pass (see mf_vegas_unweight):
    (number kept, records [min(kept, capacity), 4 + 4 n_legs]: event
    weight, x1, x2, colour-flow index, momenta)."""
    nl = proc.info["n_legs"]
    cap = n_events if capacity is None else capacity
    rec = np.zeros((max(cap, 0), 4 + 4 * nl))
    nacc = C.c_int64()
    st = L.lib().mf_vegas_unweight(grid.handle, proc.handle, n_events, seed, subprocess, _PREC[precision], w_max,
                                   lhe.handle if lhe else None, rec.ctypes.data_as(C.POINTER(C.c_double)), cap,
                                   C.byref(nacc), _stream_ptr(stream))
    L.check(st, "mf_vegas_unweight")
    return nacc.value, rec[:min(nacc.value, cap)]


def unweight_channel(grid: "Vegas", proc: "Process", channel: int, n_events: int, seed: int, w_max: float,
                     precision="mixed", lhe: LheWriter = None, capacity=None, stream=None):
    """Hit-or-miss unweighted events of one pass of phase-space channel
    `channel` through its grid (see mf_vegas_unweight_channel); returns as
    unweight."""
    nl = proc.info["n_legs"]
    cap = n_events if capacity is None else capacity
    rec = np.zeros((max(cap, 0), 4 + 4 * nl))
    nacc = C.c_int64()
    st = L.lib().mf_vegas_unweight_channel(grid.handle, proc.handle, channel, n_events, seed, _PREC[precision],
                                           w_max, lhe.handle if lhe else None,
                                           rec.ctypes.data_as(C.POINTER(C.c_double)), cap, C.byref(nacc),
                                           _stream_ptr(stream))
    L.check(st, "mf_vegas_unweight_channel")
    return nacc.value, rec[:min(nacc.value, cap)]


def channel_max_weights(proc: "Process", n_events, stream=None):
    """Largest |w| of each channel's points in the last mf_vegas_iterate_channels
    pass of n_events[k] points per channel."""
    k = len(n_events)
    N = (C.c_int64 * k)(*[int(v) for v in n_events])
    out = (C.c_double * k)()
    L.check(L.lib().mf_process_channel_max_weights(proc.handle, N, k, out, _stream_ptr(stream)),
            "mf_process_channel_max_weights")
    return [float(v) for v in out]


OBSERVABLE_KINDS = {"pt": L.MF_OBS_PT, "y": L.MF_OBS_RAPIDITY, "eta": L.MF_OBS_PSEUDORAPIDITY}


def observables(grid: "Vegas", proc: "Process", n_events: int, seed: int, obs, precision="mixed", subprocess=0,
                stream=None, channel=None):
    """Weighted histograms of one pass (see mf_vegas_observables; with a
    channel, mf_vegas_observables_channel).  obs: list of (kind, leg, nbins,
    lo, hi), kind "pt", "y" or "eta"; returns one (sigma, error, counts) per
    observable, sigma and error in pb per bin."""
    arr = (L.mf_observable * len(obs))()
    for a, (kind, leg, nbins, lo, hi) in zip(arr, obs):
        a.kind, a.leg, a.nbins, a.lo, a.hi = OBSERVABLE_KINDS[kind], leg, nbins, lo, hi
    nb = sum(o[2] for o in obs)
    sig, err = np.zeros(nb), np.zeros(nb)
    cnt = np.zeros(nb, dtype=np.int64)
    bufs = (sig.ctypes.data_as(C.POINTER(C.c_double)), err.ctypes.data_as(C.POINTER(C.c_double)),
            cnt.ctypes.data_as(C.POINTER(C.c_int64)), _stream_ptr(stream))
    if channel is None:
        L.check(L.lib().mf_vegas_observables(grid.handle, proc.handle, n_events, seed, subprocess, _PREC[precision],
                                             len(obs), arr, *bufs), "mf_vegas_observables")
    else:
        L.check(L.lib().mf_vegas_observables_channel(grid.handle, proc.handle, channel, n_events, seed,
                                                     _PREC[precision], len(obs), arr, *bufs),
                "mf_vegas_observables_channel")
    out, o = [], 0
    for kind, leg, nbins, lo, hi in obs:
        out.append((sig[o:o + nbins], err[o:o + nbins], cnt[o:o + nbins]))
        o += nbins
    return out


def read_weights(proc: "Process", idx):
    """Weights w = f J_V of the given point indices of the last Vegas pass."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    w = np.zeros(idx.shape[0])
    L.check(L.lib().mf_process_read_weights(proc.handle, idx.ctypes.data_as(C.POINTER(C.c_int64)), idx.shape[0],
                                            w.ctypes.data_as(C.POINTER(C.c_double))), "mf_process_read_weights")
    return w


def max_weight(proc: "Process", stream=None) -> float:
    w = C.c_double()
    L.check(L.lib().mf_process_max_weight(proc.handle, C.byref(w), _stream_ptr(stream)), "mf_process_max_weight")
    return w.value


class Batch:
    """Several processes in one persistent kernel (see mf_batch_create)."""

    def __init__(self, procs, precision="mixed"):
        self.procs = list(procs)            # keeps the processes alive
        k = len(self.procs)
        arr = (C.c_void_p * k)(*[p.handle.value for p in self.procs])
        h = C.c_void_p()
        L.check(L.lib().mf_batch_create(arr, k, _PREC[precision], C.byref(h)), "mf_batch_create")
        self.handle = h

    def iterate(self, grids, n_events, seed: int, refine=True, stream=None, graph=False):
        """One iteration of every subprocess; graph=True replays a captured CUDA graph."""
        k = len(self.procs)
        G = (C.c_void_p * k)(*[g.handle.value for g in grids])
        N = (C.c_int64 * k)(*n_events)
        out = (L.mf_iter_result * k)()
        fn = L.lib().mf_batch_iterate_graph if graph else L.lib().mf_batch_iterate
        st = fn(self.handle, G, N, seed, 1 if refine else 0, out, _stream_ptr(stream))
        L.check(st, "mf_batch_iterate_graph" if graph else "mf_batch_iterate", allow=(L.MF_OK, L.MF_ENAN))
        return [_result(r) for r in out]

    def info(self):
        k = len(self.procs)
        order = (C.c_int32 * k)()
        regs = C.c_int32()
        ms = C.c_double()
        L.check(L.lib().mf_batch_get_info(self.handle, order, C.byref(regs), C.byref(ms)), "mf_batch_get_info")
        return {"order": list(order), "regs": regs.value, "last_kernel_ms": ms.value}

    def close(self):
        if self.handle:
            L.lib().mf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- autograd
def integrand_with_grad(proc: "Process", x, params=None):
    """f(x) as a differentiable torch function.

    x: CUDA float64 [ndim, n] (may require grad); params: optional float64
    tensor [m_t, alpha_s] (values must be those the process was built with)
    that receives d(sum w f)/d(m_t, alpha_s) on backward.  The backward pass
    uses the derivatives mf_grad computes in the forward call.
    """
    import torch

    class _F(torch.autograd.Function):
        @staticmethod
        def forward(ctx, xin, prm):
            f, dp, dx = proc.grad(xin.detach().contiguous(), with_dx=True)
            ctx.save_for_backward(dp, dx)
            return f

        @staticmethod
        def backward(ctx, gout):
            dp, dx = ctx.saved_tensors
            gx = dx * gout[None, :] if ctx.needs_input_grad[0] else None
            gp = None
            if ctx.needs_input_grad[1]:
                gp = (dp * gout[None, :]).sum(dim=1).to(torch.float64)
            return gx, gp

    if params is None:
        params = torch.zeros(2, dtype=torch.float64, device=x.device)
    return _F.apply(x, params)
