"""CPU checks of the C-ABI library: it builds, loads and exports every function the headers declare."""
import ctypes
import glob
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(tufrg_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1710_08830_gb300 import build
    return build.build()


def test_library_exports_every_declared_function(libpath):
    declared = _declared()
    assert "tufrg_init_model" in declared and "tufrg_rhs" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = sorted(declared - exported)
    assert not missing, f"declared but not exported: {missing}"


def test_library_loads_and_binding_matches(libpath):
    from paper_1710_08830_gb300 import _lib
    L = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(L, name)
    assert set(_lib.EXPORTS) <= _declared()


def test_null_arguments_are_rejected_without_a_gpu(libpath):
    """Argument checks happen before any CUDA call."""
    from paper_1710_08830_gb300 import _lib
    L = _lib.lib()
    h = ctypes.c_void_p()
    assert L.tufrg_init_model(None, None, ctypes.byref(h)) == 1      # TUFRG_EINVAL
    assert L.tufrg_dims(None, None, None, None, None, None) == 1
    assert L.tufrg_rhs(None, 1.0, None, 3, None) == 1
    assert L.tufrg_last_error(None) == b"model handle is NULL"
    # every other entry point taking a model or network handle, and the NULL-buffer cases of the free functions
    i, d = ctypes.c_int(), ctypes.c_double()
    ll = ctypes.c_longlong()
    calls = {
        "tufrg_model_info": (None, None, None, None), "tufrg_loop_momenta": (None, ctypes.byref(i)),
        "tufrg_symmetry_info": (None, ctypes.byref(i), ctypes.byref(d), ctypes.byref(d)),
        "tufrg_deltas": (None, None), "tufrg_gather_table": (None, 0, None, 0, ctypes.byref(i)),
        "tufrg_bands": (None, None, None), "tufrg_loops": (None, 1.0, 3, None),
        "tufrg_project": (None, None, 3, None, None), "tufrg_rhs_host": (None, 1.0, None, 3, None),
        "tufrg_rhs_host_batch": (None, 0, None, None, 3, None), "tufrg_band_basis": (None, None, None),
        "tufrg_flow": (None, None, None, None), "tufrg_flow_batch": (None, 1, None, None),
        "tufrg_set_surrogate": (None, None, None, None, None, 1e-3, 0, None),
        "tufrg_surrogate_stats": (None, ctypes.byref(ll), ctypes.byref(ll), ctypes.byref(ll)),
        "tufrg_timing_begin": (None,), "tufrg_timing_end": (None, None, 0, None, None),
        "tufrg_set_device_error": (None, 1), "tufrg_loops_info": (None, ctypes.byref(i)),
        "tufrg_loop_tiles": (None, ctypes.byref(i), ctypes.byref(i), None, 0),
        "tufrg_products_tiles": (None, ctypes.byref(i), ctypes.byref(i), None, 0),
        "tufrg_flow_start": (None, None), "tufrg_flow_step": (None, None), "tufrg_flow_amax_channels": (None, None),
        "tufrg_flow_end": (None, None, None), "tufrg_flow_save": (None, None, 0),
        "tufrg_flow_resume": (None, None, None, 0),
        "tufrg_shard_classes": (None, ctypes.byref(i), None), "tufrg_form_factors": (None, None, None),
        "tufrg_irrep_basis": (None, None, 0, None), "tufrg_rhs_shard_transform": (None, None, 1, None, 3, None),
        "tufrg_rhs_shard_finish": (None, 0.1, None, 1, None, None, 3, None),
        "tufrg_mlp_create": (4, 8, 1, 2, 0, None, None), "tufrg_mlp_get_params": (None, None),
        "tufrg_mlp_set_params": (None, None), "tufrg_mlp_forward": (None, None, 1, None),
        "tufrg_mlp_gradients": (None, None, None, 1, None, None), "tufrg_mlp_train_step": (None, None, None, 1, 1e-3, None),
        "tufrg_round_f32": (None, None, 5, None), "tufrg_widen_f64": (None, None, 5, None),
        "tufrg_loops_noalloc": (4, 2, None, None, 0.0, 0.1, 5, None, 3, None, None),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == 1, name                # TUFRG_EINVAL
    assert L.tufrg_flow_checkpoint_bytes(None) == 0
    assert L.tufrg_mlp_num_params(None) == -1
    assert L.tufrg_mlp_last_error(None) == b"network handle is NULL"
    L.tufrg_free(None)
    L.tufrg_mlp_free(None)


def test_host_allocation_failure_is_a_status_not_an_exception(libpath):
    """A host allocation that fails inside an entry point returns TUFRG_ENOMEM instead of throwing across the C
    boundary (which would end the caller's process).  tufrg_mlp_create's initial weights (64 layers of width 4096,
    4.2 GB) are allocated on the host before any CUDA call, here in a child process whose address space is limited
    to 1 GB more than it already maps; no device is touched."""
    code = r"""
import ctypes, resource, sys
L = ctypes.CDLL(sys.argv[1])
L.tufrg_mlp_last_error.restype = ctypes.c_char_p
vm = 0
for line in open("/proc/self/status"):
    if line.startswith("VmSize:"):
        vm = int(line.split()[1]) * 1024
resource.setrlimit(resource.RLIMIT_AS, (vm + (1 << 30), resource.getrlimit(resource.RLIMIT_AS)[1]))
out = ctypes.c_void_p()
st = L.tufrg_mlp_create(16, 4096, 64, 16, ctypes.c_ulonglong(0), None, ctypes.byref(out))
msg = L.tufrg_mlp_last_error(out) if out.value else b""
print(st, msg.decode())
"""
    r = subprocess.run([sys.executable, "-c", code, libpath], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    st, msg = r.stdout.strip().split(" ", 1)
    assert int(st) == 2 and msg.startswith("host allocation failed"), r.stdout


def test_bad_descriptors_are_rejected_before_device_use(libpath):
    import numpy as np
    from paper_1710_08830_gb300 import _lib, inputs
    L = _lib.lib()
    spec = inputs.rashba_hubbard(Lq=6, nc=2, n_ff=5)
    hopR = np.ascontiguousarray(spec.hop_R, np.int32)
    hopt = np.ascontiguousarray(spec.hop_t, np.complex128)
    V0 = np.ascontiguousarray(spec.V0, np.complex128)

    def init(ff, **kw):
        ff = np.ascontiguousarray(ff, np.int32)
        f = dict(n_s=2, n_hop=hopR.shape[0], hop_R=hopR.ctypes.data, hop_t=hopt.ctypes.data, mu=-0.9, filling=0.0,
                 T_mu=0.02, V0=V0.ctypes.data, n_ff=ff.shape[0], ff_R=ff.ctypes.data, Lq=6, nc=2, precision=0)
        f.update(kw)
        d = _lib.ModelDesc(**f)
        h = ctypes.c_void_p()
        st = L.tufrg_init_model(ctypes.byref(d), None, ctypes.byref(h))
        msg = L.tufrg_last_error(h).decode()
        L.tufrg_free(h)
        return st, msg

    st, msg = init(np.array([[1, 0], [0, 0]]))
    assert st == 1 and "(0,0)" in msg
    st, msg = init(np.array([[0, 0], [6, 0]]))
    assert st == 1 and "distinct" in msg
    st, msg = init(spec.ff_R, Lq=1)
    assert st == 1
    st, msg = init(spec.ff_R, precision=7)
    assert st == 1
    st, msg = init(spec.ff_R, symmetry=7)   # AUTO, OFF, STATES are 0, 1, 2
    assert st == 1 and "symmetry" in msg
    bad = hopt.copy()
    bad[0] *= 2.0   # breaks t_{-R} = t_R^dagger
    st, msg = init(spec.ff_R, hop_t=bad.ctypes.data)
    assert st == 1 and "Hermitian" in msg
    # every remaining check of the descriptor, each before the first CUDA call
    EINVAL, ENOTSUP = 1, 8
    cases = [
        (dict(n_s=0), EINVAL, "n_s"), (dict(n_s=9), EINVAL, "n_s"), (dict(n_s=3), ENOTSUP, "n_s = 2, 4, 6"),
        (dict(n_hop=0), EINVAL, "hopping"), (dict(V0=None), EINVAL, "V0"), (dict(n_ff=0), EINVAL, "bond set"),
        (dict(nc=0), EINVAL, "Lq >= 2"), (dict(Lq=64, nc=65), EINVAL, "fine mesh"),
        (dict(products=9), EINVAL, "products"), (dict(loops=3), EINVAL, "loops backend"),
        (dict(basis=2), EINVAL, "basis"), (dict(filling=0.5, T_mu=0.0), EINVAL, "T_mu"),
        (dict(regulator=7), EINVAL, "regulator"), (dict(regulator=1, T_reg=0.0), EINVAL, "T_reg"),
        (dict(regulator=1, T_reg=float("nan")), EINVAL, "T_reg"),
        (dict(n_hop=hopR.shape[0] - 1), EINVAL, "t_{-R}"),      # the last hop loses its partner
    ]
    for kw, want, text in cases:
        st, msg = init(spec.ff_R, **kw)
        assert st == want and text in msg, (kw, st, msg)
    # the largest fine mesh (Lq nc = 4096) passes the size check and stops at the next one
    st, msg = init(spec.ff_R, Lq=64, nc=64, precision=7)
    assert st == EINVAL and "precision" in msg
