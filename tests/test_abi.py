"""The C-ABI library builds, loads and exports every entry point that
include/sparkling.h declares; ctypes structs match the C layout; argument
validation rejects bad calls before any CUDA call (no GPU needed)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sparkling.h")

needs_nvcc = pytest.mark.skipif(
    shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
    reason="nvcc not available")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SPARKLING_API\s+[\w\s\*]*?\b(sparkling_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2108_02991_gb300 import build
    build.build()
    import paper_2108_02991_gb300 as sp
    return sp


@needs_nvcc
def test_exports_every_declared_symbol(lib):
    decl = declared_symbols()
    assert len(decl) >= 10
    L = lib.lib()
    for name in decl:
        assert hasattr(L, name), f"{name} declared in sparkling.h but not exported"
    assert sorted(lib.ABI_SYMBOLS) == decl
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = sorted(set(re.findall(r"\bT (sparkling_\w+)", out)))
    assert exported == decl, "the library exports exactly the declared ABI"


@needs_nvcc
def test_binding_constants_match_the_header(lib):
    """Every integer #define of sparkling.h that the binding also names
    (without the SPARKLING_ prefix) has the same value there; the kernel
    kinds are the binding's KERNEL_NAMES in header order."""
    sp = lib
    text = open(HEADER).read()
    consts = dict((n, int(v)) for n, v in re.findall(r"#define SPARKLING_(\w+)\s+(-?\d+)", text))
    shared = [n for n in consts if hasattr(sp, n)]
    assert len(shared) >= 20
    for n in shared:
        assert getattr(sp, n) == consts[n], f"SPARKLING_{n}"
    kinds = sorted((v, n) for n, v in consts.items()
                   if n.startswith("KERNEL_") and n != "KERNEL_COUNT")
    assert [n[len("KERNEL_"):].lower() for _, n in kinds] == list(sp.KERNEL_NAMES)
    assert consts["KERNEL_COUNT"] == len(sp.KERNEL_NAMES)


@needs_nvcc
def test_struct_layout_matches_c(lib, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sparkling.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(sparkling_grid), offsetof(sparkling_grid, n), sizeof(sparkling_proj),"
        "offsetof(sparkling_proj, pin), offsetof(sparkling_proj, pin_index),"
        "offsetof(sparkling_proj, n_iter), offsetof(sparkling_proj, check_every),"
        "offsetof(sparkling_grid, hi), sizeof(sparkling_schedule),"
        "offsetof(sparkling_schedule, n_git), offsetof(sparkling_schedule, beta_factor));"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    G, P, S = lib.Grid, lib.Proj, lib.Schedule
    want = [ctypes.sizeof(G), G.n.offset, ctypes.sizeof(P), P.pin.offset, P.pin_index.offset,
            P.n_iter.offset, P.check_every.offset, G.hi.offset, ctypes.sizeof(S), S.n_git.offset,
            S.beta_factor.offset]
    assert got == want


@needs_nvcc
def test_version_and_context_without_gpu(lib):
    assert "sm_103a" in lib.sparkling_version()
    ctx = lib.sparkling_create(0)       # makes no CUDA call
    assert lib.sparkling_launch_count(ctx) == 0
    lib.sparkling_destroy(ctx)
    with pytest.raises(lib.SparklingError) as e:
        lib.Context(-1)
    assert e.value.code == lib.E_INVAL


@needs_nvcc
def test_argument_validation_before_any_cuda_call(lib):
    """Every bad argument is refused with SPARKLING_E_INVAL and a message;
    none of these calls reaches the CUDA runtime."""
    L = lib.lib()
    ctx = lib.sparkling_create(0)
    h = ctx.handle
    dummy = ctypes.c_void_p(0x1000)     # never dereferenced: validation fails first
    g = lib.Grid()
    g.rho, g.lo, g.hi = dummy, -0.5, 0.5
    for a in range(3):
        g.n[a] = 8
    p = lib.make_proj(0.01, 0.001)

    def grad(K=dummy, kd=0, N=100, grid=g, acc=0, G=dummy, gd=0):
        return L.sparkling_grad(h, K, kd, N, ctypes.byref(grid) if grid is not None else None,
                                acc, G, gd, None, None, None)

    cases = {
        "K is NULL": grad(K=None),
        "dtype": grad(kd=7),
        "N = 1": grad(N=1),
        "N = 0": grad(N=0),
        "acc": grad(acc=5),
        "grid is NULL": grad(grid=None),
        "G is NULL": grad(G=None),
        "G dtype": grad(gd=2),
        "N beyond the 32-bit sample index": grad(N=(1 << 31)),
        "N far beyond": grad(N=(1 << 40)),
    }
    bad = lib.Grid(); bad.rho, bad.lo, bad.hi = dummy, 0.5, -0.5
    for a in range(3):
        bad.n[a] = 4
    cases["lo < hi"] = grad(grid=bad)
    bad2 = lib.Grid(); bad2.rho, bad2.lo, bad2.hi = dummy, -0.5, 0.5
    bad2.n[0], bad2.n[1], bad2.n[2] = 5000, 4, 4
    cases["nx exceeds"] = grad(grid=bad2)
    bad3 = lib.Grid(); bad3.rho, bad3.lo, bad3.hi = dummy, -0.5, 0.5
    bad3.n[0], bad3.n[1], bad3.n[2] = 4, 0, 4
    cases["n[1]"] = grad(grid=bad3)
    for what, code in cases.items():
        assert code == lib.E_INVAL, what
    # shot shapes at and beyond the limits
    assert L.sparkling_step(h, dummy, 0, 4, 65537, ctypes.byref(g), 0, 1e-3, ctypes.byref(p),
                            None) == lib.E_INVAL          # Ns > 65536
    assert L.sparkling_step(h, dummy, 0, (1 << 40), 8, ctypes.byref(g), 0, 1e-3, ctypes.byref(p),
                            None) == lib.E_INVAL          # Nc * Ns too large
    # projection parameters
    def proj(Nc=4, Ns=8, pr=p):
        return L.sparkling_project(h, dummy, 0, Nc, Ns, ctypes.byref(pr) if pr else None, None, None)
    assert proj(Nc=0) == lib.E_INVAL
    assert proj(Ns=0) == lib.E_INVAL
    assert proj(pr=None) == lib.E_INVAL
    for field, value in (("alpha", 0.0), ("beta", -1.0), ("box", 0.0), ("n_iter", -1),
                         ("pin_index", 8), ("alpha", float("nan"))):
        q = lib.make_proj(0.01, 0.001)
        setattr(q, field, value)
        assert proj(pr=q) == lib.E_INVAL, field
    q = lib.make_proj(0.01, 0.001, tol=1e-9, check_every=0)
    assert proj(pr=q) == lib.E_INVAL
    q = lib.make_proj(0.01, 0.001, tol=1e-9, margin=1.5)
    assert proj(pr=q) == lib.E_INVAL
    msg = lib.sparkling_last_error(ctx)
    assert "margin" in msg
    assert L.sparkling_grad(None, dummy, 0, 10, ctypes.byref(g), 0, dummy, 0, None, None, None) == lib.E_INVAL
    assert "ctx" in lib.sparkling_last_error(None)
    # pinned tile shapes
    assert L.sparkling_set_shape(None, 1, 0) == lib.E_INVAL
    assert L.sparkling_set_shape(h, 0, 0) == lib.E_INVAL          # pack has no shapes
    assert L.sparkling_set_shape(h, 1, 3) == lib.E_INVAL
    assert L.sparkling_set_shape(h, 2, 4) == lib.E_INVAL
    assert L.sparkling_set_shape(h, 2, -2) == lib.E_INVAL
    for k, v in ((1, 2), (1, -1), (2, 2), (2, 3), (2, -1)):
        assert L.sparkling_set_shape(h, k, v) == lib.OK
    # projection arithmetic, wait budget, memory cap (host-side settings)
    assert L.sparkling_set_projection(h, 2) == lib.E_INVAL
    assert L.sparkling_set_step_path(None, 0) == lib.E_INVAL
    assert L.sparkling_set_step_path(h, 3) == lib.E_INVAL
    assert L.sparkling_set_step_path(h, -1) == lib.E_INVAL
    for v in (lib.STEP_ENGINE, lib.STEP_KERNELS, lib.STEP_AUTO):
        assert L.sparkling_set_step_path(h, v) == lib.OK
    assert L.sparkling_set_projection(None, 0) == lib.E_INVAL
    for m in (lib.PROJECTION_MIXED, lib.PROJECTION_FP64):
        assert L.sparkling_set_projection(h, m) == lib.OK
    assert L.sparkling_set_wait_budget(h, (1 << 40) + 1) == lib.E_INVAL
    assert L.sparkling_set_wait_budget(h, 0) == lib.OK          # no CUDA call before first use
    assert L.sparkling_set_wait_budget(h, -1) == lib.OK
    assert L.sparkling_set_memory_limit(h, -5) == lib.E_INVAL
    assert L.sparkling_set_memory_limit(h, 1 << 20) == lib.OK
    assert L.sparkling_set_memory_limit(h, 0) == lib.OK
    # the plain FP64-accumulate mode is an accepted accumulation mode
    assert grad(acc=lib.ACC_FP64_PAIR, K=None) == lib.E_INVAL and "K is NULL" in \
        lib.sparkling_last_error(ctx)
    assert grad(acc=3) == lib.E_INVAL and "acc" in lib.sparkling_last_error(ctx)
    # attraction mode
    assert L.sparkling_set_attraction(h, 7) == lib.E_INVAL
    assert L.sparkling_set_attraction(h, lib.ATTRACTION_FIELD) == lib.OK
    assert L.sparkling_attraction_field(h, None, None) == lib.E_INVAL
    assert L.sparkling_attraction_field(h, ctypes.byref(bad), None) == lib.E_INVAL
    assert L.sparkling_set_attraction(h, lib.ATTRACTION_DIRECT) == lib.OK
    # regularised kernel
    for eps in (-1.0, float("nan"), float("inf"), 1e4):
        assert L.sparkling_set_regularisation(h, eps) == lib.E_INVAL, eps
    assert L.sparkling_set_regularisation(h, 0.02) == lib.OK
    assert L.sparkling_set_regularisation(h, 0.0) == lib.OK
    # driver: schedule and level checks
    def opt(sc, Nc=4, Ns=8):
        return L.sparkling_optimize(h, dummy, 0, Nc, Ns, ctypes.byref(g), ctypes.byref(p), 0,
                                    ctypes.byref(sc) if sc is not None else None, None, None)
    assert opt(None) == lib.E_INVAL
    for field, value in (("eta", 0.0), ("eta", float("inf")), ("eta_min", 0.0),
                         ("eta_max", 1e-20), ("alpha_factor", -2.0), ("n_git", -1),
                         ("n_fixed", -3)):
        sc = lib.make_schedule(1e-3, 10)
        setattr(sc, field, value)
        assert opt(sc) == lib.E_INVAL, field
    sc = lib.make_schedule(1e-3, 10)
    def multi(start, Ns=64):
        return L.sparkling_multires(h, dummy, 0, 4, Ns, ctypes.byref(g), ctypes.byref(p), 0,
                                    ctypes.byref(sc), start, None, None, None)
    assert multi(-1) == lib.E_INVAL
    assert multi(3, Ns=36) == lib.E_INVAL          # 36 is not a multiple of 8
    assert L.sparkling_upsample(h, dummy, dummy, 0, 4, 8, None) == lib.E_INVAL   # overlap
    assert L.sparkling_upsample(h, dummy, None, 0, 4, 8, None) == lib.E_INVAL
    assert L.sparkling_upsample(h, dummy, ctypes.c_void_p(0x100000), 0, 0, 8, None) == lib.E_INVAL
    assert lib.sparkling_launch_count(ctx) == 0
    lib.sparkling_destroy(ctx)


@needs_nvcc
def test_split_host_logic(lib, tmp_path):
    """The even split of (tile, unit) work over persistent CTAs: every unit is
    covered exactly once, CTA ranges are contiguous, and the number of CTAs
    touching a tile never exceeds the partial-slot count."""
    src = tmp_path / "split.cpp"
    src.write_text(r'''
#include <cstdio>
#include "kernels.h"
using namespace sparkling;
int main() {
  long bad = 0, checked = 0;
  const long tiles_l[] = {1, 2, 3, 7, 19, 256, 1000};
  const long per_l[] = {1, 2, 3, 10, 33, 1024, 16384};
  const long ctas_l[] = {1, 2, 5, 100, 152, 456, 1000, 5000};
  for (long T : tiles_l) for (long P : per_l) for (long C : ctas_l) {
    Split s = make_split(T, P, C);
    if (s.ctas > s.units || s.ctas < 1) ++bad;
    long prev = 0;
    for (long c = 0; c < s.ctas; ++c) {
      long b = split_begin(s, c), e = split_begin(s, c + 1);
      if (b != prev || e < b) ++bad;
      prev = e;
      for (long u = b; u < e; ++u) if (split_cta_of(s, u) != c) ++bad;
    }
    if (prev != s.units) ++bad;
    for (long t = 0; t < T; ++t) {
      long lo = split_cta_of(s, t * P), hi = split_cta_of(s, (t + 1) * P - 1);
      if (hi - lo + 1 > s.slots) ++bad;
    }
    ++checked;
  }
  std::printf("%ld %ld\n", checked, bad);
  return bad != 0;
}
''')
    exe = tmp_path / "split"
    cuda_inc = "/usr/local/cuda/include"
    subprocess.run(["g++", "-std=c++17", "-I", os.path.join(ROOT, "paper_2108_02991_gb300", "csrc"),
                    "-I", cuda_inc, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    checked, bad = map(int, r.stdout.split())
    assert checked == 7 * 7 * 8 and bad == 0


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    """No fallback: if the shared library is absent, loading raises."""
    import paper_2108_02991_gb300 as sp
    monkeypatch.setattr(sp, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(sp, "_lib_handle", None)
    with pytest.raises(ImportError):
        sp.lib()


@needs_nvcc
def test_triangle_pair_numbering(tmp_path):
    """Tile pairs (I, J), I <= J, numbered row by row: tri_pair inverts the
    numbering exactly (every pair of small triangles, sampled large ones)."""
    src = tmp_path / "tri.cpp"
    src.write_text(r'''
#include <cstdio>
#include "kernels.h"
using namespace sparkling;
int main() {
  long bad = 0, checked = 0;
  for (long T = 1; T <= 60; ++T) {
    long u = 0;
    for (long I = 0; I < T; ++I)
      for (long J = I; J < T; ++J, ++u) {
        int64_t i, j; tri_pair(u, T, i, j);
        if (i != I || j != J) ++bad;
        ++checked;
      }
    if (u != tri_count(T)) ++bad;
  }
  const long big[] = {1024, 10240, 100000, 2097151};
  for (long T : big) {
    const long U = tri_count(T);
    for (long k = 0; k < 200000; ++k) {
      const long u = (long)((double)k / 200000 * U) + (k % 7);
      if (u >= U) continue;
      int64_t i, j; tri_pair(u, T, i, j);
      if (i < 0 || j < i || j >= T || tri_row_start(i, T) + (j - i) != u) ++bad;
      ++checked;
    }
    int64_t i, j; tri_pair(U - 1, T, i, j);
    if (i != T - 1 || j != T - 1) ++bad;
  }
  std::printf("%ld %ld\n", checked, bad);
  return bad != 0;
}
''')
    exe = tmp_path / "tri"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I",
                    os.path.join(ROOT, "paper_2108_02991_gb300", "csrc"), "-I",
                    "/usr/local/cuda/include", str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    checked, bad = map(int, r.stdout.split())
    assert checked > 500000 and bad == 0
