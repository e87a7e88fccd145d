"""C-ABI checks that need no GPU: the library loads, exports every symbol
declared in include/hsvd.h, rejects invalid arguments before touching the
device, and its host-side schedule helpers agree with the tree and Jacobi
orderings they describe."""
import ctypes
import os
import re

import pytest

from paper_1710_02812_gb300 import hsvd
from oracle import hmat as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(hsvd.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return hsvd.lib()


def declared_functions():
    with open(os.path.join(ROOT, "include", "hsvd.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hsvd_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "hsvd_plan" in names and "hsvd_run" in names and "hsvd_factors" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(hsvd.EXPORTED)


def test_error_strings(lib):
    for code in range(6):
        assert hsvd.error_string(code)
    assert hsvd.error_string(0) == "success"


@pytest.mark.parametrize("count", [1, 2, 3, 5, 7, 8, 64, 65, 1000])
def test_tree_levels_match_merge_schedule(lib, count):
    assert hsvd.hsvd_tree_levels(count) == len(H.tree_schedule(count))
    assert hsvd.hsvd_tree_levels(0) == -1


@pytest.mark.parametrize("n", [2, 4, 6, 20, 64, 128, 256])
def test_jacobi_round_robin_covers_each_pair_once(lib, n):
    seen = set()
    for r in range(n - 1):
        used = set()
        for s in range(n // 2):
            p, q = hsvd.hsvd_jacobi_pair(n, r, s)
            assert 0 <= p < n and 0 <= q < n and p != q
            assert p not in used and q not in used       # disjoint within a round
            used.update((p, q))
            pair = (min(p, q), max(p, q))
            assert pair not in seen                      # once per sweep
            seen.add(pair)
    assert len(seen) == n * (n - 1) // 2


def test_register_core_ordering_covers_each_column_pair_once_per_sweep(lib):
    """The ordering of the register-resident cluster cores: two CTAs of 16
    blocks of 8 columns, 15 + 8 + 8 rounds and two exchanges of a quarter per
    sweep.  Every pair of the 256 columns meets exactly once; in every round
    the 8 warps of a CTA hold its 16 blocks once each; the 8 pairs of a step
    use 16 distinct register columns."""
    order = hsvd.hsvd_jacobi_block_order
    for kind, nsteps in ((0, 8), (1, 7)):
        seen = set()
        for t in range(nsteps):
            cols = [c for p in range(8) for c in order(1, kind, t, p)]
            assert sorted(cols) == list(range(16))
            for p in range(8):
                a, b = order(1, kind, t, p)
                if kind == 0:
                    assert a < 8 <= b
                else:
                    assert (a < 8) == (b < 8)
                seen.add((min(a, b), max(a, b)))
        want = 64 if kind == 0 else 2 * 28
        assert len(seen) == want
    g = [[16 * me + p for p in range(16)] for me in range(2)]   # global block at each position
    met = {}

    def meet(u, v):
        key = (min(u, v), max(u, v))
        assert u != v and key not in met
        met[key] = 1

    for me in range(2):   # pairs inside each block
        for p in range(16):
            for t in range(7):
                for q in range(4):
                    a, b = order(1, 1, t, q)
                    meet(8 * g[me][p] + a, 8 * g[me][p] + b)
    for ph in range(3):
        if ph == 1:
            for k in range(8):
                g[0][8 + k], g[1][k] = g[1][k], g[0][8 + k]
        if ph == 2:
            for k in range(8):
                g[0][8 + k], g[1][8 + k] = g[1][8 + k], g[0][8 + k]
        for r in range(15 if ph == 0 else 8):
            held = [blk for w in range(8) for blk in order(0, ph, r, w)]
            assert sorted(held) == list(range(16))
            for me in range(2):
                for w in range(8):
                    a, b = order(0, ph, r, w)
                    for t in range(8):
                        for p in range(8):
                            i, j = order(1, 0, t, p)
                            meet(8 * g[me][a] + i, 8 * g[me][b] + (j - 8))
    assert len(met) == 256 * 255 // 2
    for args in [(2, 0, 0, 0), (0, 3, 0, 0), (0, 0, 15, 0), (0, 1, 8, 0), (0, 0, 0, 8), (1, 1, 7, 0),
                 (1, 0, 8, 0), (1, 2, 0, 0)]:
        with pytest.raises(hsvd.HsvdError):
            order(*args)


def test_jacobi_pair_rejects_bad_arguments(lib):
    for args in [(3, 0, 0), (4, 3, 0), (4, 0, 2), (0, 0, 0)]:
        with pytest.raises(hsvd.HsvdError):
            hsvd.hsvd_jacobi_pair(*args)


def _plan_code(lib, batch=1, m=(64,), n=(64,), br=16, bc=16, mode=0, param=4.0, cap=8, tree=0, prec=1, dt=1,
               opts=None):
    h = ctypes.c_void_p(1234)
    ma = (ctypes.c_int64 * max(1, len(m)))(*m)
    na = (ctypes.c_int64 * max(1, len(n)))(*n)
    code = lib.hsvd_plan(ctypes.byref(h), batch, ma, na, br, bc, mode, param, cap, tree, prec, dt, opts)
    return code, h


@pytest.mark.parametrize("kw", [
    dict(batch=0), dict(m=(0,)), dict(n=(-3,)), dict(br=0), dict(bc=-1), dict(mode=7),
    dict(mode=0, param=0.0), dict(mode=0, param=2.5), dict(mode=1, param=1.0), dict(mode=1, param=0.0),
    dict(mode=2, param=1.5), dict(mode=2, param=0.0), dict(cap=0), dict(cap=257), dict(tree=5),
    dict(prec=0, dt=1), dict(prec=1, dt=0), dict(prec=1, dt=2), dict(prec=2, dt=0), dict(prec=9),
    dict(param=float("nan")),
])
def test_plan_rejects_invalid_arguments_without_a_device(lib, kw):
    code, h = _plan_code(lib, **kw)
    assert code == hsvd.HSVD_EINVAL
    assert h.value is None  # out set to NULL on failure


def test_plan_rejects_bad_options(lib):
    o = hsvd.Options(-1, 0, 0.0, 0, 0, 0)
    code, _ = _plan_code(lib, opts=ctypes.byref(o))
    assert code == hsvd.HSVD_EINVAL
    o = hsvd.Options(0, -5, 0.0, 0, 0, 0)
    code, _ = _plan_code(lib, opts=ctypes.byref(o))
    assert code == hsvd.HSVD_EINVAL


def test_null_handles_are_rejected(lib):
    assert lib.hsvd_plan(None, 1, None, None, 1, 1, 0, 1.0, 1, 0, 1, 1, None) == hsvd.HSVD_EINVAL
    assert lib.hsvd_run(None, None, None, None) == hsvd.HSVD_EINVAL
    assert lib.hsvd_run_host(None, None, None, None) == hsvd.HSVD_EINVAL
    assert lib.hsvd_status_query(None, 0, None) == hsvd.HSVD_EINVAL
    assert lib.hsvd_factors(None, 0, None, None, 0, None, None, 0, 0, None) == hsvd.HSVD_EINVAL
    assert lib.hsvd_workspace_bytes(None) == 0
    assert lib.hsvd_launches_per_run(None) == -1
    assert lib.hsvd_last_error(None) == b""
    assert lib.hsvd_refine(None, 1, 1e-3, None, None, None) == hsvd.HSVD_EINVAL
    assert lib.hsvd_gram(None, 4, 4, 4, 1, None, 4, None) == hsvd.HSVD_EINVAL
    lib.hsvd_destroy(None)


def test_valid_plan_without_device_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    code, h = _plan_code(lib)
    assert code == hsvd.HSVD_ECUDA
    assert h.value is None


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libhsvd.so the binding raises on first use; nothing falls back
    to a CPU implementation."""
    monkeypatch.setattr(hsvd, "LIB_PATH", str(tmp_path / "libhsvd.so"))
    monkeypatch.setattr(hsvd, "_lib_handle", None)
    with pytest.raises(RuntimeError, match="no fallback"):
        hsvd.lib()
    with pytest.raises(RuntimeError, match="no fallback"):
        hsvd.Plan(64, 64, 32, 32, "fixed_k", 4, prec="f32")
    with pytest.raises(RuntimeError, match="no fallback"):
        hsvd.hsvd_tree_levels(5)


def test_plain_c_client_builds_and_runs_host_entry_points(lib, tmp_path):
    """The header is plain C99: a C client compiles with -pedantic -Werror,
    links against libhsvd.so and runs the entry points that need no device."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = tmp_path / "c_abi_client"
    libdir = os.path.dirname(hsvd.LIB_PATH)
    cmd = [cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_client.c"), "-o", str(exe), "-L", libdir, "-lhsvd",
           "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)


def _planless(m, n, in_dtype="f32", prec="f32", kcap=4):
    """A Plan object with the planned sizes but no device plan: any library
    call would fail, so an error here must come from the binding's checks."""
    p = object.__new__(hsvd.Plan)
    p.m, p.n, p.in_dtype, p.prec, p.kcap = list(m), list(n), in_dtype, prec, kcap
    p._h = None
    return p


def test_binding_rejects_inputs_the_kernels_would_overrun():
    import numpy as np
    import torch
    p = _planless([6, 5], [4, 3])
    good = [torch.zeros(6, 4), torch.zeros(5, 3)]
    with pytest.raises(ValueError, match="the plan holds 2"):
        hsvd.check_inputs(good[:1], p.m, p.n, "f32", device=False)
    with pytest.raises(ValueError, match="shape"):
        hsvd.check_inputs([torch.zeros(6, 4), torch.zeros(4, 3)], p.m, p.n, "f32", device=False)
    with pytest.raises(TypeError, match="dtype"):
        hsvd.check_inputs([torch.zeros(6, 4, dtype=torch.float64), good[1]], p.m, p.n, "f32", device=False)
    with pytest.raises(TypeError, match="dtype"):  # an f32 buffer for an f64 plan is half the bytes
        hsvd.check_inputs(good, p.m, p.n, "f64", device=False)
    with pytest.raises(ValueError, match="contiguous"):
        hsvd.check_inputs([torch.zeros(4, 6).t(), good[1]], p.m, p.n, "f32", device=False)
    with pytest.raises(TypeError, match="2-D"):
        hsvd.check_inputs([torch.zeros(24), good[1]], p.m, p.n, "f32", device=False)
    hsvd.check_inputs(good, p.m, p.n, "f32", device=False)                 # host inputs are fine
    hsvd.check_inputs([np.zeros((6, 4), np.float32), np.zeros((5, 3), np.float32)], p.m, p.n, "f32",
                      device=False)
    wide = torch.zeros(6, 10)[:, 2:6]                                        # ld 10 > n 4: allowed
    hsvd.check_inputs([wide, good[1]], p.m, p.n, "f32", device=False)
    with pytest.raises(TypeError, match="dtype"):                          # numpy has no bf16
        hsvd.check_inputs([np.zeros((6, 4), np.float32), np.zeros((5, 3), np.float32)], p.m, p.n, "bf16",
                          device=False)
    # run() checks before any library call; host tensors are not device memory
    with pytest.raises(ValueError, match="CUDA tensor"):
        p.run(good)
    with pytest.raises(TypeError, match="CUDA tensor"):
        p.run([np.zeros((6, 4), np.float32), np.zeros((5, 3), np.float32)])
    with pytest.raises(ValueError, match="shape"):
        p.run_host([np.zeros((5, 4), np.float32), np.zeros((5, 3), np.float32)])


def test_binding_rejects_factor_outputs_too_small_or_of_the_wrong_type():
    import torch
    p = _planless([6], [4], kcap=3)
    with pytest.raises(TypeError, match="CUDA tensor"):
        p.factors_device(torch.zeros(3, 6), None, None)
    with pytest.raises(TypeError, match="CUDA tensor"):
        hsvd.check_factor_outputs(None, torch.zeros(3), None, 3, 6, 4, "f32")
    hsvd.check_factor_outputs(None, None, None, 3, 6, 4, "f32")             # nothing requested


def test_gram_binding_rejects_mismatched_buffers():
    import torch
    x = torch.zeros(8, 5)
    with pytest.raises(ValueError, match="5 x 5"):
        hsvd.hsvd_gram(x, torch.zeros(4, 4))
    with pytest.raises(TypeError, match="float32"):
        hsvd.hsvd_gram(x, torch.zeros(5, 5, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA"):
        hsvd.hsvd_gram(x, torch.zeros(5, 5))


def test_noalloc_binding_rejects_buffers_the_kernels_would_overrun():
    """hsvd_block_svd_noalloc receives raw pointers: the binding checks every
    buffer before the call (shape, type, strides, sizes, device)."""
    import torch
    m, n, k = 12, 10, 4

    def args(**over):
        a = dict(A=torch.zeros(m, n), m=m, n=n, k=k, U=torch.zeros(k, m), S=torch.zeros(k),
                 rank=torch.zeros(1, dtype=torch.int32), flags=torch.zeros(1, dtype=torch.int32))
        a.update(over)
        return a

    chk = hsvd.check_noalloc_args
    chk(**args(), require_cuda=False)                                        # well-formed
    chk(**args(flags=None), require_cuda=False)                              # flags are optional
    chk(**args(A=torch.zeros(m, 16)[:, :n]), require_cuda=False)             # row stride 16 > n
    with pytest.raises(ValueError, match="CUDA tensor"):                     # host memory
        chk(**args())
    with pytest.raises(ValueError, match="shape"):
        chk(**args(A=torch.zeros(m + 1, n)), require_cuda=False)
    with pytest.raises(TypeError, match="float32"):
        chk(**args(A=torch.zeros(m, n, dtype=torch.float64)), require_cuda=False)
    with pytest.raises(ValueError, match="contiguous"):
        chk(**args(A=torch.zeros(n, m).t()), require_cuda=False)            # column stride != 1
    with pytest.raises(ValueError, match="contiguous"):
        chk(**args(lda=n - 1), require_cuda=False)
    with pytest.raises(ValueError, match="at least 48"):
        chk(**args(U=torch.zeros(k, m - 1)), require_cuda=False)             # fewer than k * ldu
    with pytest.raises(ValueError, match="ldu"):
        chk(**args(ldu=m - 1), require_cuda=False)
    with pytest.raises(ValueError, match="at least 4"):
        chk(**args(S=torch.zeros(k - 1)), require_cuda=False)
    with pytest.raises(TypeError, match="int32"):
        chk(**args(rank=torch.zeros(1, dtype=torch.int64)), require_cuda=False)
    with pytest.raises(TypeError, match="int32"):
        chk(**args(flags=torch.zeros(1)), require_cuda=False)
    with pytest.raises(TypeError, match="torch tensor"):
        chk(**args(S=[0.0] * k), require_cuda=False)
    # the public entry point checks before any library call
    with pytest.raises(ValueError, match="CUDA tensor"):
        hsvd.hsvd_block_svd_noalloc(torch.zeros(m, n), m, n, k, 1, torch.zeros(k, m), torch.zeros(k),
                                    torch.zeros(1, dtype=torch.int32))
