"""GB300-native leading-order integrand library (MadFlow method, arXiv:2106.10279).

The compute path is libmadflow_gb.so (C ABI in include/madflow_gb.h): fused
CUDA kernels specialised per process at run time for sm_103a.  This package
holds the thin Python binding (``api``), the host-side process builder
(``process``) and the build script (``build``).  There is no CPU fallback:
using the binding without the built library raises.
"""
import os as _os

_HERE = _os.path.dirname(_os.path.abspath(__file__))
# compiled process kernels are cached here unless the caller chose a directory
_os.environ.setdefault("MF_JIT_CACHE", _os.path.join(_HERE, "_build", "jit_cache"))
if _os.environ["MF_JIT_CACHE"]:
    _os.makedirs(_os.environ["MF_JIT_CACHE"], exist_ok=True)
