"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every function include/nefty.h declares, the ctypes structures match
the header, and argument validation behaves as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nefty.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2603_11045_gb300 import build, _native
    build.build()
    return _native.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nefty_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "nefty_forward" in names and "nefty_adjoint_grad" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in nefty.h but not exported"


def test_struct_fields_match_header():
    from paper_2603_11045_gb300 import _native as N
    src = open(HEADER).read()
    structs = (("nefty_problem", N.nefty_problem), ("nefty_stats", N.nefty_stats), ("nefty_job", N.nefty_job),
               ("nefty_job_result", N.nefty_job_result), ("nefty_serve_config", N.nefty_serve_config),
               ("nefty_field_desc", N.nefty_field_desc))
    sizes = {"int32_t": 4, "double": 8, "int64_t": 8, "uint64_t": 8,
             "nefty_problem": ctypes.sizeof(N.nefty_problem)}
    for struct, cls in structs:
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + struct + ";", src, flags=re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        decl = []
        for line in body.split(";"):
            line = line.strip()
            if not line:
                continue
            words = line.replace("*", " * ").split()
            pointer = "*" in words
            words = [w for w in words if w not in ("*", "const")]
            typ, names = words[0], " ".join(words[1:])
            for nm in names.split(","):
                decl.append((nm.strip(), "pointer" if pointer else typ))
        assert [d[0] for d in decl] == [f[0] for f in cls._fields_], struct
        for (nm, typ), (cn, ct) in zip(decl, cls._fields_):
            assert ctypes.sizeof(ct) == (8 if typ == "pointer" else sizes[typ]), (struct, nm)


def _problem(**kw):
    from paper_2603_11045_gb300.solver import Problem
    args = dict(nx=4, ny=3, nz=2, nt=5)
    args.update(kw)
    return Problem(**args).to_c()


@pytest.mark.parametrize("bad", [dict(nx=0), dict(nt=0), dict(dx=0.0), dict(dz=-1.0), dict(dt=0.0),
                                 dict(bc=7), dict(obs_face=2), dict(robin_h=-0.1), dict(rtol=-1.0),
                                 dict(max_iter=-1), dict(ckpt_every=-2), dict(loss_scale=-1.0), dict(extrap=5), dict(extrap=-2), dict(jacobi_k=-1), dict(jacobi_k=100001),
                                 dict(nx=2048, ny=2048, nz=512), dict(dx=float("nan"))])
def test_problem_validation_rejects(lib, bad):
    p = _problem(**bad)
    assert lib.nefty_problem_check(ctypes.byref(p)) == 1
    assert lib.nefty_last_error(None)


def test_problem_validation_accepts(lib):
    for kw in (dict(), dict(bc=1, obs_face=1, robin_h=0.5, prec="fp64", ckpt_every=3)):
        p = _problem(**kw)
        assert lib.nefty_problem_check(ctypes.byref(p)) == 0


def test_create_without_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.nefty_create(ctypes.byref(h), 0, 0)
    assert st == 4 and not h.value
    assert b"device" in lib.nefty_last_error(None)


def test_status_strings(lib):
    assert lib.nefty_status_string(0) == b"NEFTY_OK"
    assert lib.nefty_status_string(3) == b"NEFTY_ENOTCONV"


def test_debug_barrier_fault_needs_a_handle(lib):
    """The fault-injection hook validates its handle on the host (no device work)."""
    assert lib.nefty_debug_barrier_fault(None, 1, 0) == 1   # NEFTY_EINVAL
    assert b"handle" in lib.nefty_last_error(None)


def _field(**kw):
    from paper_2603_11045_gb300.field import FieldSpec
    args = dict(nx=8, ny=6, nz=4, n_freq=5, width=128, depth=3, skip_layer=2)
    args.update(kw)
    return FieldSpec(**args).to_c()


def test_field_param_count_and_validation(lib):
    """nefty_field_param_count follows the packed layout of nefty.h (W_0 [W x 6F],
    b_0, W_l [W x in_l], b_l, w_out, b_out) and returns 0 for an invalid
    descriptor; keep_activations is a 0/1 switch that leaves the layout alone."""
    F, W, L, s = 5, 128, 3, 2
    want = W * 6 * F + W + sum(W * (W + 6 * F if l == s else W) + W for l in range(1, L)) + W + 1
    for keep in (0, 1):
        d = _field(keep_activations=bool(keep))
        assert d.keep_activations == keep
        assert lib.nefty_field_param_count(ctypes.byref(d)) == want
    d = _field()
    d.keep_activations = 2
    assert lib.nefty_field_param_count(ctypes.byref(d)) == 0
    for bad in (dict(width=100), dict(depth=0), dict(precision=2), dict(skip_layer=3), dict(n_freq=0),
                dict(freq_lo=0.0), dict(alpha_min=2.0, alpha_max=1.0)):
        assert lib.nefty_field_param_count(ctypes.byref(_field(**bad))) == 0, bad


def test_field_activation_reuses_of_null_handle(lib):
    assert lib.nefty_field_activation_reuses(None) == 0
