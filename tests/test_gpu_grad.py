"""Gradients (mf_grad) against finite differences and the oracle.

* df/dx_j against central differences of mf_integrand (h = 1e-6);
* df/dm_t against central differences over processes built with
  m_t (1 +- 1e-3) (relative <= 1e-4), excluding points whose cut or threshold
  status differs between m_t +- h (the moving cut boundary is not part of the
  pathwise derivative);
* df/dalpha_s = k f / alpha_s against central differences in alpha_s;
* df/dm_t and df/dx_j against Richardson-extrapolated central differences of
  the oracle (relative <= 1e-6) and against the oracle's forward-mode dual
  numbers (relative <= 1e-9);
* the value it returns against the oracle with the FP64 parity bound;
* the summed pathwise dsigma/dm_t against the finite difference of sigma over
  the same points, and the boundary term reported separately (gg->tt~g and
  gg->tt~gg), with dsigma/dalpha_s = k sigma / alpha_s;
* the torch.autograd wrapper.
"""
import math

import numpy as np
import pytest

import workloads as W
from _tolerance import fp64_tolerance, relerr

pytestmark = pytest.mark.gpu

NAMES = ["ee_mumu", "gg_ttx", "uux_ttx", "gg_ttxg", "uux_ttxg", "gg_ttxgg"]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    return torch


@pytest.fixture(scope="module")
def procs(torch_cuda):
    from paper_2106_10279_gb300 import api
    cache = {}

    def get(name, **kw):
        key = (name, tuple(sorted(kw.items())))
        if key not in cache:
            cache[key] = api.Process.from_workload(W.WORKLOADS[name], **kw)
        return cache[key]
    return get


def _f(torch, proc, x):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = proc.integrand(xd, "fp64").cpu().numpy()
    return out


def _grad(torch, proc, x):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    f, dp, dx = proc.grad(xd)
    torch.cuda.synchronize()
    return f.cpu().numpy(), dp.cpu().numpy(), dx.cpu().numpy()


@pytest.mark.parametrize("name", NAMES)
def test_grad_value_equals_integrand(torch_cuda, procs, oracle_processes, name):
    # the value mf_grad returns is the FP64 integrand: against the oracle with
    # the parity bound of mf_integrand, and zero (with zero derivatives)
    # exactly where mf_integrand is zero
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    x = W.uniform_points(wl.ndim, 200, 41)
    p = procs(name)
    f, dp, dx = _grad(torch_cuda, p, x)
    ref, tol = fp64_tolerance(Integrand(wl, process=oracle_processes(name)), x)
    assert np.array_equal(f == 0, _f(torch_cuda, p, x) == 0)
    assert np.array_equal(f == 0, ref == 0)
    r = relerr(f, ref)
    assert np.all(r <= tol), (name, r.max(), int(np.argmax(r / tol)))
    nz = ref != 0
    assert np.all(dp[:, ~nz] == 0) and np.all(dx[:, ~nz] == 0)


@pytest.mark.parametrize("name,n", [("ee_mumu", 64), ("gg_ttx", 64), ("uux_ttx", 64), ("gg_ttxg", 48),
                                    ("uux_ttxg", 48), ("gg_ttxgg", 24)])
def test_dx_matches_central_differences(torch_cuda, procs, name, n):
    wl = W.WORKLOADS[name]
    x = np.clip(W.uniform_points(wl.ndim, n, 42), 1e-3, 1 - 1e-3)
    p = procs(name)
    f, dp, dx = _grad(torch_cuda, p, x)
    h = 1e-6
    for j in range(wl.ndim):
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        fp, fm = _f(torch_cuda, p, xp), _f(torch_cuda, p, xm)
        same = (fp != 0) & (fm != 0) & (f != 0)
        fd = (fp - fm) / (2 * h)
        scale = np.abs(fd) + np.abs(f)          # derivative relative to the value's scale
        err = np.abs(dx[j] - fd)[same] / scale[same]
        assert err.max() < 1e-5, (name, j, err.max())


@pytest.mark.parametrize("name,n", [("gg_ttx", 200), ("uux_ttx", 100), ("gg_ttxg", 100), ("uux_ttxg", 80),
                                    ("gg_ttxgg", 40)])
def test_dmt_matches_central_differences(torch_cuda, procs, name, n):
    wl = W.WORKLOADS[name]
    x = W.uniform_points(wl.ndim, n, 43)
    h = 1e-3 * wl.m_top
    f, dp, dx = _grad(torch_cuda, procs(name), x)
    fp = _f(torch_cuda, procs(name, m_top=wl.m_top + h), x)
    fm = _f(torch_cuda, procs(name, m_top=wl.m_top - h), x)
    same = (fp != 0) & (fm != 0) & (f != 0)
    assert same.sum() > 0.5 * n
    fd = (fp - fm) / (2 * h)
    # relative to |f|/m_t: the natural scale of a mass derivative
    err = np.abs(dp[0] - fd)[same] / (np.abs(fd) + np.abs(f) / wl.m_top)[same]
    assert err.max() < 1e-4, (name, err.max())


@pytest.mark.parametrize("name", ["gg_ttx", "gg_ttxg", "uux_ttxg", "gg_ttxgg"])
def test_dalphas_is_exact(torch_cuda, procs, name):
    wl = W.WORKLOADS[name]
    x = W.uniform_points(wl.ndim, 100, 44)
    f, dp, dx = _grad(torch_cuda, procs(name), x)
    k = {"gg_ttx": 2, "gg_ttxg": 3, "uux_ttxg": 3, "gg_ttxgg": 4}[name]
    nz = f != 0
    assert np.allclose(dp[1][nz], k * f[nz] / wl.alpha_s, rtol=1e-14)
    h = 1e-3 * wl.alpha_s
    fp = _f(torch_cuda, procs(name, alpha_s=wl.alpha_s + h), x)
    fm = _f(torch_cuda, procs(name, alpha_s=wl.alpha_s - h), x)
    fd = (fp - fm) / (2 * h)
    assert np.max(np.abs(dp[1][nz] / fd[nz] - 1)) < 1e-5


@pytest.mark.parametrize("name,n", [("gg_ttx", 12), ("gg_ttxg", 8)])
def test_grad_matches_oracle_richardson(torch_cuda, procs, name, n):
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    x = W.uniform_points(wl.ndim, n, 45)
    f, dp, dx = _grad(torch_cuda, procs(name), x)

    def fo(mt):
        return Integrand(wl, m_top=mt)(x)

    def rich(fun, x0, h):
        d1 = (fun(x0 + h) - fun(x0 - h)) / (2 * h)
        d2 = (fun(x0 + h / 2) - fun(x0 - h / 2)) / h
        return d2 + (d2 - d1) / 3
    mt = wl.m_top
    # step 1e-3 m_t: the extrapolated difference is then exact to ~1e-10
    # (1e-2 m_t leaves O(1e-6) truncation near threshold)
    ref = rich(fo, mt, 1e-3 * mt)
    nz = f != 0
    err = np.abs(dp[0] - ref)[nz] / (np.abs(ref) + np.abs(f) / mt)[nz]
    assert err.max() < 1e-6, err.max()
    I = Integrand(wl)
    for j in (0, wl.ndim - 1):
        def fx(v, j=j):
            xx = x.copy()
            xx[j] = v
            return I(xx)
        ref = rich(fx, x[j], 1e-4)
        err = np.abs(dx[j] - ref)[nz] / (np.abs(ref) + np.abs(f))[nz]
        assert err.max() < 1e-6, (j, err.max())


@pytest.mark.parametrize("name,n", [("gg_ttxg", 20000), ("gg_ttxgg", 20000)])
def test_summed_dsigma_dmt_and_boundary_term(torch_cuda, procs, name, n):
    # pathwise estimator of dsigma/dm_t = mean df/dm_t against the finite
    # difference of the same-point mean, restricted to points that keep their
    # cut status; the full finite difference also contains the boundary term
    # (points entering or leaving the cuts and the threshold as m_t moves)
    wl = W.WORKLOADS[name]
    x = W.uniform_points(wl.ndim, n, 46)
    h = 1e-3 * wl.m_top
    f, dp, dx = _grad(torch_cuda, procs(name), x)
    fp = _f(torch_cuda, procs(name, m_top=wl.m_top + h), x)
    fm = _f(torch_cuda, procs(name, m_top=wl.m_top - h), x)
    same = (fp != 0) & (fm != 0) & (f != 0)
    pathwise = np.mean(np.where(same, dp[0], 0.0))
    fd_same = np.mean(np.where(same, (fp - fm) / (2 * h), 0.0))
    fd_all = np.mean((fp - fm) / (2 * h))
    assert abs(pathwise / fd_same - 1) < 1e-4, (pathwise, fd_same)
    boundary = fd_all - fd_same
    print(f"{name}: dsigma/dm_t pathwise {pathwise:.6g} pb/GeV, finite difference {fd_all:.6g}, "
          f"boundary term {boundary:.3g} ({boundary / fd_all:.2%})")
    # at pT(g) > 20 GeV alone the moving boundary is a small effect; with
    # Delta R(g,g) > 0.4 as well the few points that cross it sit next to the
    # collinear enhancement, so the finite-difference boundary term is a
    # large, high-variance sum of rare heavy points: reported, not bounded
    if name == "gg_ttxg":
        assert abs(boundary) < 0.05 * abs(fd_all)
    # dsigma/dalpha_s = k sigma / alpha_s over the same points
    k = {"gg_ttxg": 3, "gg_ttxgg": 4}[name]
    assert np.mean(dp[1]) == pytest.approx(k * np.mean(f) / wl.alpha_s, rel=1e-13)


def test_autograd_wrapper(torch_cuda, procs):
    torch = torch_cuda
    from paper_2106_10279_gb300 import api
    wl = W.GG_TTX
    p = procs("gg_ttx")
    x = torch.from_numpy(W.uniform_points(wl.ndim, 500, 47)).cuda().requires_grad_(True)
    prm = torch.tensor([wl.m_top, wl.alpha_s], dtype=torch.float64, device="cuda", requires_grad=True)
    f = api.integrand_with_grad(p, x, prm)
    sigma = f.mean()
    sigma.backward()
    f2, dp, dx = p.grad(x.detach())
    assert torch.allclose(x.grad, dx / 500, rtol=1e-14, atol=0)
    assert torch.allclose(prm.grad, dp.mean(dim=1), rtol=1e-12)
    assert prm.grad[1].item() == pytest.approx(2 * sigma.item() / wl.alpha_s, rel=1e-12)


@pytest.mark.parametrize("name,n", [("ee_mumu", 30), ("gg_ttx", 40), ("uux_ttx", 40), ("gg_ttxg", 20),
                                    ("uux_ttxg", 20), ("gg_ttxgg", 32)])
def test_grad_matches_oracle_dual_numbers(torch_cuda, procs, oracle_processes, name, n):
    # both sides exact to rounding: the GPU's forward tangents plus
    # hand-written adjoints against the oracle's forward-mode dual numbers
    from oracle.integrand import Integrand
    wl = W.WORKLOADS[name]
    I = Integrand(wl, process=oracle_processes(name))
    x = np.clip(W.uniform_points(wl.ndim, n, 48), 1e-3, 1 - 1e-3)
    f, dp, dx = _grad(torch_cuda, procs(name), x)
    fo, dxo, dmo = I.gradient(x)
    nz = fo != 0
    assert np.array_equal(f == 0, fo == 0)
    assert nz.sum() >= min(16, n // 2), nz.sum()
    err = np.abs(dx - dxo)[:, nz] / (np.abs(dxo) + np.abs(fo))[:, nz]
    assert err.max() < 1e-9, err.max()
    mt = wl.m_top
    errm = np.abs(dp[0] - dmo)[nz] / (np.abs(dmo) + np.abs(fo) / mt)[nz]
    assert errm.max() < 1e-9, errm.max()
