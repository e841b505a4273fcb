"""The C-ABI boundary without a GPU: the library loads, exports every symbol
include/lassogs.h and include/lista.h declare, and its host-only logic behaves
as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_1505_03410_gb300.build import build
    build()
    import paper_1505_03410_gb300 as p
    p.load()
    return p


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b((?:lasso|lista)_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(pkg):
    lib = ctypes.CDLL(pkg.lassogs.LIB_PATH)
    declared = _declared_functions()
    assert set(declared) >= set(pkg.EXPORTED) | set(pkg.lista.EXPORTED)
    assert {n for n in declared if n.startswith("lista_")} == set(pkg.lista.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_default_opts(pkg):
    o = pkg.lasso_default_opts()
    assert (o.screen_period, o.dual_point, o.xtr_scope, o.warm_start) == (10, 0, 0, 1)
    assert o.max_epochs == 100000 and o.gap_tol_rel == 1e-6 and o.gemm_dtype == pkg.LASSO_BF16
    assert (o.batch_ctas_per_sm, o.gemm_tile_n, o.batch_group, o.screen_rule, o.refined_radius) == (0, 0, 0, 0, 0)
    assert o.enet_alpha == 1.0


def test_lambda_grid_matches_oracle(pkg):
    """Sec. 3.3 grid: the library's host helper and the oracle's agree bit for bit."""
    for T, d in [(100, 3.0), (50, 2.0), (30, 2.0), (1, 3.0), (2, 0.5)]:
        np.testing.assert_array_equal(pkg.lasso_lambda_grid(T, d), oracle.lambda_ratios(T, d))
    with pytest.raises(pkg.LassoError) as e:
        pkg.lasso_lambda_grid(0, 3.0)
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG
    with pytest.raises(pkg.LassoError):
        pkg.lasso_lambda_grid(10, -1.0)


def test_workspace_size(pkg):
    a = pkg.lasso_path_workspace_size(500, 50000, pkg.LASSO_F32)
    b = pkg.lasso_path_workspace_size(500, 50000, pkg.LASSO_F64)
    assert 0 < a < b
    assert pkg.lasso_path_workspace_size(2049, 10, pkg.LASSO_F32) == 0
    assert pkg.lasso_path_workspace_size(0, 10, pkg.LASSO_F32) == 0
    assert pkg.lasso_path_workspace_size(10, 0, pkg.LASSO_F32) == 0
    assert pkg.lasso_path_workspace_size(10, 10, pkg.LASSO_BF16) == 0
    bad = pkg.lasso_default_opts(screen_period=0)
    assert pkg.lasso_path_workspace_size(10, 10, pkg.LASSO_F32, bad) == 0


def _call(pkg, **kw):
    args = dict(X=0x10000, x_dtype=pkg.LASSO_F32, n=8, p=16, ldx=8, y=0x20000, lambda_ratios=0x30000, T=4,
                beta0=None, opts=pkg.lasso_default_opts(), beta_out=0x40000, mask_out=None, stats=0x50000,
                workspace=0x100000, workspace_bytes=1 << 30, stream=None)
    args.update(kw)
    return pkg.lasso_path(**args)


@pytest.mark.parametrize("kw,status", [
    (dict(X=None), 1), (dict(y=None), 1), (dict(stats=None), 1), (dict(n=0), 1), (dict(n=2049), 1),
    (dict(p=0), 1), (dict(T=0), 1), (dict(ldx=7), 1), (dict(ldx=10), 1), (dict(X=0x10008), 1),
    (dict(x_dtype=2), 1), (dict(workspace=None), 3), (dict(workspace=0x100010), 3),
    (dict(workspace_bytes=16), 3),
])
def test_argument_errors(pkg, kw, status):
    """Invalid arguments are rejected on the host before any CUDA call."""
    with pytest.raises(pkg.LassoError) as e:
        _call(pkg, **kw)
    assert e.value.status == status
    assert pkg.lasso_last_error() != ""


@pytest.mark.parametrize("field,value", [("screen_period", 0), ("dual_point", 2), ("xtr_scope", -1),
                                         ("warm_start", 3), ("max_epochs", -1), ("gap_tol_rel", -1.0),
                                         ("gemm_dtype", 7), ("batch_ctas_per_sm", 3), ("gemm_tile_n", 96),
                                         ("batch_group", 65), ("batch_group", -1), ("screen_rule", 2),
                                         ("refined_radius", 2), ("enet_alpha", 0.0), ("enet_alpha", 1.5),
                                         ("enet_alpha", float("nan"))])
def test_option_errors(pkg, field, value):
    o = pkg.lasso_default_opts(**{field: value})
    with pytest.raises(pkg.LassoError) as e:
        _call(pkg, opts=o)
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG


def test_product_has_no_cpu_fallback(pkg, tmp_path):
    """Loading from a path without the library fails loudly."""
    import importlib
    mod = importlib.import_module("paper_1505_03410_gb300.lassogs")
    saved = mod._lib
    try:
        mod._lib = None
        with pytest.raises(RuntimeError):
            mod.load(str(tmp_path / "missing.so"))
    finally:
        mod._lib = saved


def test_lista_host_checks(pkg):
    """Sizes and NULL arguments of the learned-warm-start entry points are
    rejected on the host, before any CUDA call."""
    L = pkg.lista
    assert L.lista_workspace_size(0, 10, 8, 4) == 0
    assert L.lista_workspace_size(10, 10, 0, 4) == 0
    assert L.lista_workspace_size(10, 10, 65, 4) == 0
    # the cache of a training batch: L x B x (n + 2p) floats at least
    assert L.lista_workspace_size(300, 10000, 8, 256) >= 8 * 256 * (300 + 2 * 10000) * 4
    with pytest.raises(pkg.LassoError) as e:
        L.lista_forward(None, 10, 20, 10, None, None, None, 8, None, 10, 4, None, 0, None, 0, None)
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG
    with pytest.raises(pkg.LassoError) as e:
        L.lista_backward(None, 10, 20, 10, None, None, None, 0, 4, None, None, None, None, None, None, None, 0, None)
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG
    with pytest.raises(pkg.LassoError) as e:
        L.lista_adam(None, None, None, None, 10, 1, 1e-3, 0.9, 0.999, 1e-8, None)
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG
    with pytest.raises(pkg.LassoError) as e:
        L.lista_adam(1, 1, 1, 1, 10, 0, 1e-3, 0.9, 0.999, 1e-8, None)  # t must be >= 1
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG


def test_tune_host_checks(pkg):
    """The autotuner's sizes and arguments are checked on the host."""
    assert pkg.lasso_batch_tune_candidates() == 11
    assert pkg.lasso_batch_tune_workspace_size(100, 1000, 0, 5) == 0
    assert pkg.lasso_batch_tune_workspace_size(100, 1000, 16, 5) >= 16 * 5 * 1000 * 8
    tuned = pkg.LassoOpts()
    with pytest.raises(pkg.LassoError) as e:  # sample > B
        pkg.lasso_batch_tune(None, 100, 1000, 100, None, 100, None, 0, 4, None, 10, None, 0, None, 8, 5, tuned,
                             None, None, 0, None)
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG


def test_batch_group_needs_fp32_checks(pkg):
    """Groups of CTAs per problem run the per-CTA FP32 mode only."""
    o = pkg.lasso_default_opts(batch_group=4)  # default gemm_dtype is LASSO_BF16
    with pytest.raises(pkg.LassoError) as e:
        pkg.lasso_batch(1 << 12, 10, 20, 12, 1 << 12, 10, None, 0, 2, 1 << 12, 3, None, 0, o, 1 << 12, None,
                        1 << 12, 1 << 12, 1 << 20, None)
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG


@pytest.mark.parametrize("a", [0.0, -0.5, 1.5, float("nan")])
def test_enet_alpha_out_of_range(pkg, a):
    """The Elastic-Net's mixing a must lie in (0, 1]; the host rejects the
    rest before any CUDA call, for both solvers."""
    with pytest.raises(pkg.LassoError) as e:
        _call(pkg, opts=pkg.lasso_default_opts(enet_alpha=a))
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG
    with pytest.raises(pkg.LassoError) as e:
        pkg.lasso_batch(1 << 12, 10, 20, 12, 1 << 12, 10, None, 0, 2, 1 << 12, 3, None, 0,
                        pkg.lasso_default_opts(enet_alpha=a, gemm_dtype=pkg.LASSO_F32), 1 << 12, None,
                        1 << 12, 1 << 12, 1 << 20, None)
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG


@pytest.mark.parametrize("v", [-1, 2])
def test_lockstep_pass_out_of_range(pkg, v):
    """lockstep_pass is 0 or 1; the host rejects the rest before any CUDA
    call, and the workspace query answers 0 for it."""
    o = pkg.lasso_default_opts(lockstep_pass=v)
    with pytest.raises(pkg.LassoError) as e:
        pkg.lasso_batch(1 << 12, 10, 20, 12, 1 << 12, 10, None, 0, 2, 1 << 12, 3, None, 0, o, 1 << 12, None,
                        1 << 12, 1 << 12, 1 << 20, None)
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG
    assert "lockstep_pass" in pkg.lasso_last_error()
    assert pkg.lasso_batch_workspace_size(10, 20, 2, o) == 0


def test_pass_lockstep_workspace_holds_the_single_path_region(pkg):
    """Lockstep per pass may finish its last problems on the single path, so
    its workspace holds a single-path region (at least lasso_path's own
    workspace) on top of the per-lambda lockstep's."""
    n, p, B = 500, 3000, 40
    per_lambda = pkg.lasso_batch_workspace_size(n, p, B, pkg.lasso_default_opts(gemm_dtype=pkg.LASSO_BF16))
    per_pass = pkg.lasso_batch_workspace_size(n, p, B, pkg.lasso_default_opts(gemm_dtype=pkg.LASSO_BF16,
                                                                              lockstep_pass=1))
    single = pkg.lasso_path_workspace_size(n, p, pkg.LASSO_F32)
    assert per_lambda > 0 and single > 0
    assert per_pass >= per_lambda + single
    # the option only matters for lockstep batches
    f32 = pkg.lasso_default_opts(gemm_dtype=pkg.LASSO_F32)
    f32p = pkg.lasso_default_opts(gemm_dtype=pkg.LASSO_F32, lockstep_pass=1)
    assert pkg.lasso_batch_workspace_size(n, p, B, f32) == pkg.lasso_batch_workspace_size(n, p, B, f32p)


def test_struct_layouts_match_the_header(pkg, tmp_path):
    """The ctypes mirrors of lasso_opts and lasso_path_stats have the field
    offsets and sizes a C compiler gives the declarations in lassogs.h."""
    import ctypes
    import os
    import subprocess
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    mirrors = {"lasso_opts": pkg.LassoOpts, "lasso_path_stats": pkg.LassoPathStats}
    lines = ['#include <stdio.h>', '#include "lassogs.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            cf = "lambda" if fname == "lambda_" else fname
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {cf}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", inc, "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "lassogs.h"

int main(void) {
  lasso_opts o;
  lasso_default_opts(&o);
  double r[5];
  if (lasso_lambda_grid(5, 2.0, r) != LASSO_OK) return 1;
  printf("grid %.17g %.17g\n", r[0], r[4]);
  printf("ws %zu\n", lasso_path_workspace_size(500, 50000, LASSO_F32, &o));
  /* a host-side argument error: no device work, a message, INVALID_ARG */
  lasso_status st = lasso_path(NULL, LASSO_F32, 8, 16, 8, NULL, NULL, 4, NULL, &o, NULL, NULL, NULL, NULL, 0, NULL);
  printf("status %d %s\n", (int)st, strlen(lasso_last_error()) > 0 ? "message" : "none");
  o.screen_period = 0;
  printf("bad %zu\n", lasso_path_workspace_size(10, 10, LASSO_F32, &o));
  return 0;
}
"""


def test_c_client_links_and_calls_the_host_api(pkg, tmp_path):
    """A plain C program compiles against include/lassogs.h, links
    liblassogs.so and calls its host-only entry points: the ABI needs neither
    Python nor C++ on the caller's side."""
    import subprocess
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(pkg.lassogs.LIB_PATH)
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src),
                           "-L", libdir, "-llassogs", f"-Wl,-rpath,{libdir}"])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    grid = out[0].split()
    assert float(grid[1]) == 1.0 and float(grid[2]) == pkg.lasso_lambda_grid(5, 2.0)[4]
    assert int(out[1].split()[1]) == pkg.lasso_path_workspace_size(500, 50000, pkg.LASSO_F32)
    assert out[2] == f"status {pkg.LASSO_ERR_INVALID_ARG} message"
    assert out[3] == "bad 0"
