"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/icmpt.h declares; without a GPU it
fails loudly instead of falling back to the CPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1501_05630_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "icmpt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(icm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1501_05630_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("icm_ctx_create", "icm_batch_create", "icm_set_schedule", "icm_run_sweeps",
                 "icm_read_energies", "icm_read_observables", "icm_read_spins", "icm_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name
    nm = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (icm_\w+)", nm))
    assert set(_declared()) <= exported
    from paper_1501_05630_gb300 import icmpt
    assert set(icmpt.EXPORTS) == set(_declared())


def test_library_is_built_for_sm_103a(lib_path):
    out = subprocess.run(["cuobjdump", "--list-elf", lib_path], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_lattice_sizes_on_host(lib_path):
    from paper_1501_05630_gb300 import icmpt
    assert icmpt.lattice_size(I.SQUARE2D, 8) == (64, 128)
    assert icmpt.lattice_size(I.CUBIC3D, 8) == (512, 1536)
    assert icmpt.lattice_size(I.CHIMERA, 8) == (512, 1472)
    assert icmpt.lattice_size(I.CHIMERA, 12) == (1152, 3360)
    with pytest.raises(icmpt.IcmError):
        icmpt.lattice_size(7, 8)


def test_no_cpu_fallback_without_gpu(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1501_05630_gb300 import icmpt
    with pytest.raises(icmpt.IcmError):
        icmpt.Context(0)


def test_context_options_checked_on_host(lib_path):
    """Context options are validated before any device call; without a GPU a
    budgeted context fails loudly like a plain one."""
    import torch
    from paper_1501_05630_gb300 import icmpt
    with pytest.raises(ValueError):
        icmpt.Context(0, allocator="numpy")
    lib = ctypes.CDLL(lib_path)
    lib.icm_ctx_create_ex.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    assert lib.icm_ctx_create_ex(None, 0, None, 0, None) == -1            # ICM_ERR_ARG: no out pointer
    bad = (ctypes.c_void_p * 3)(None, None, None)                        # allocator without its functions
    h = ctypes.c_void_p()
    assert lib.icm_ctx_create_ex(ctypes.byref(h), 0, None, 0, ctypes.byref(bad)) == -1
    if not torch.cuda.is_available():
        with pytest.raises(icmpt.IcmError):
            icmpt.Context(0, hbm_budget=1 << 20)


def test_missing_library_fails_loudly(tmp_path):
    from paper_1501_05630_gb300 import icmpt
    with pytest.raises(RuntimeError):
        icmpt.load_library.__wrapped__(str(tmp_path / "nope.so")) if hasattr(icmpt.load_library, "__wrapped__") \
            else _load_fresh(icmpt, str(tmp_path / "nope.so"))


def _load_fresh(icmpt, path):
    saved = icmpt._lib
    icmpt._lib = None
    try:
        return icmpt.load_library(path)
    finally:
        icmpt._lib = saved


def test_inputs_are_deterministic_and_typed():
    a = I.couplings(100, I.GAUSS, 7, [3, 4])
    b = I.couplings(100, I.GAUSS, 7, [3, 4])
    assert a.dtype == np.float32 and np.array_equal(a, b)
    c = I.couplings(100, I.PM_J, 7, [3])
    assert c.dtype == np.int8 and set(np.unique(c)) <= {-1, 1}
    s = I.initial_spins(64, 8, 1, [0, 1])
    assert s.shape == (2, 8, 64) and set(np.unique(s)) <= {-1, 1}
    T = I.ladder(0.2, 2.0, 24)
    assert T[0] == 0.2 and abs(T[-1] - 2.0) < 1e-12 and np.all(np.diff(T) > 0)
    assert int(np.sum(T <= 1.0)) == 17


class _FakeTensor:
    """Just the attributes energies_static inspects (no device memory)."""

    def __init__(self, shape, dtype, index=0, cuda=True, contiguous=True):
        import types
        self.shape, self.dtype, self.is_cuda = tuple(shape), dtype, cuda
        self.device = types.SimpleNamespace(index=index)
        self._contiguous = contiguous

    def is_contiguous(self):
        return self._contiguous


def test_energies_static_checks_shapes_dtypes_and_device():
    """Wrong dtypes, shapes or devices are refused with ValueError before the
    library is called (it would read or write past the caller's buffers)."""
    from paper_1501_05630_gb300.icmpt import _check_static_args
    N, Nb, n, r = 512, 1536, 3, 48
    ok = dict(couplings=_FakeTensor((n, Nb), "torch.float32"), spins=_FakeTensor((n, r, N), "torch.int8"),
              out=_FakeTensor((n, r), "torch.float64"))
    assert _check_static_args(0, N, Nb, I.GAUSS, **ok) == (n, r)
    pmj = dict(ok, couplings=_FakeTensor((n, Nb), "torch.int8"))
    assert _check_static_args(0, N, Nb, I.PM_J, **pmj) == (n, r)
    bad = [
        (I.GAUSS, dict(ok, couplings=_FakeTensor((n, Nb), "torch.int8"))),      # +-J couplings passed as Gaussian
        (I.PM_J, ok),                                                          # float couplings passed as +-J
        (I.GAUSS, dict(ok, couplings=_FakeTensor((n, Nb - 1), "torch.float32"))),
        (I.GAUSS, dict(ok, spins=_FakeTensor((n, r, N - 1), "torch.int8"))),
        (I.GAUSS, dict(ok, spins=_FakeTensor((n, r, N), "torch.float32"))),
        (I.GAUSS, dict(ok, out=_FakeTensor((n, r), "torch.float32"))),
        (I.GAUSS, dict(ok, out=_FakeTensor((n, r + 1), "torch.float64"))),
        (I.GAUSS, dict(ok, out=_FakeTensor((n, r), "torch.float64", index=1))),   # another device
        (I.GAUSS, dict(ok, spins=_FakeTensor((n, r, N), "torch.int8", cuda=False))),
        (I.GAUSS, dict(ok, spins=_FakeTensor((n, r, N), "torch.int8", contiguous=False))),
    ]
    for dis, kw in bad:
        with pytest.raises(ValueError):
            _check_static_args(0, N, Nb, dis, **kw)
