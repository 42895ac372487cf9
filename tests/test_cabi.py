"""The C-ABI library builds, loads without a GPU and exports every declared symbol (CPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "mm.h")) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\**\s+\**(mm_[a-z_A-Z0-9]+)\s*\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("mm_plan", "mm_apply_A", "mm_precond", "mm_build_coarse", "mm_solve", "mm_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1408_3048_gb300 import build, mm
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(mm.EXPORTS) == _declared()
    assert lib.mm_version
    fn = lib.mm_version
    fn.restype = ctypes.c_char_p
    assert b"sm_103a" in fn()


def test_null_arguments_are_rejected_without_a_gpu():
    from paper_1408_3048_gb300 import mm
    L = mm.lib()
    h = ctypes.c_void_p()
    assert L.mm_plan(ctypes.byref(h), None, 0, 0, None, None, 0, None, None, 0, None) == mm.MM_ERR_ARG
    assert h.value is None
    assert L.mm_apply_A(None, 0, None, None) == mm.MM_ERR_ARG
    n = ctypes.c_int32(-1)
    assert L.mm_solve_history(None, 0, None, ctypes.byref(n)) == mm.MM_ERR_ARG
    L.mm_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without libmm.so every entry point raises instead of computing
    from paper_1408_3048_gb300 import mm
    monkeypatch.setattr(mm, "LIBPATH", str(tmp_path / "absent" / "libmm.so"))
    monkeypatch.setattr(mm, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        mm.lib()
    with pytest.raises(RuntimeError):
        mm.mm_version()


def test_invalid_plans_are_rejected_on_the_host():
    # argument checks that run before any device work (CPU): bad ncomp, lambda >= the
    # shortest interval, non-increasing offsets
    import numpy as np
    from paper_1408_3048_gb300 import mm
    L = mm.lib()
    pix = np.zeros(100, dtype=np.int32)
    off = np.array([0, 50, 100], dtype=np.int64)
    ipsd = np.zeros(2, dtype=np.int32)
    psd = (mm.mm_psd * 1)(mm.mm_psd(1.0, 1.0, 1.0))

    def plan(lam=10, ncomp=1, pix_=pix, off_=off):
        o = mm.mm_opts(ncomp=ncomp, lambda_=lam, window=0, fsamp=100.0, rcond_min=1e-6)
        h = ctypes.c_void_p()
        st = L.mm_plan(ctypes.byref(h), pix_.ctypes.data, pix_.size, 4, None, off_.ctypes.data, off_.size - 1,
                       ipsd.ctypes.data, psd, 1, ctypes.byref(o))
        if h.value:
            L.mm_destroy(h)
        return st

    assert plan(ncomp=2) == mm.MM_ERR_ARG
    assert plan(lam=50) == mm.MM_ERR_ARG
    assert plan(off_=np.array([0, 60, 50, 100], dtype=np.int64)) == mm.MM_ERR_ARG


def test_binding_rejects_mistyped_or_missized_arrays_before_any_call():
    # plain pointers carry no type or size: the binding checks both against the plan before
    # the C call (a float32 buffer passed for doubles would be read past its end).  A Plan
    # shell without a library handle shows that nothing reaches the library or the GPU.
    torch = pytest.importorskip("torch")
    from paper_1408_3048_gb300 import mm
    p = mm.Plan.__new__(mm.Plan)
    p._torch, p.handle, p.n, p.nt, p.npsd = torch, None, 12, 40, 1
    f64, f32 = torch.float64, torch.float32
    cases = [
        (lambda: p.solve(torch.zeros(40, dtype=f32)), TypeError),
        (lambda: p.solve(torch.zeros(39, dtype=f64)), ValueError),
        (lambda: p.solve(torch.zeros(40, dtype=f64), out=torch.zeros(12, dtype=f32)), TypeError),
        (lambda: p.rhs(np.zeros(40, dtype=np.float32)), TypeError),
        (lambda: p.apply_A(torch.zeros(12, dtype=f64), mm.MM_FP32), TypeError),
        (lambda: p.apply_A(torch.zeros(13, dtype=f64)), ValueError),
        (lambda: p.gather(torch.zeros(40, dtype=f64)), ValueError),
        (lambda: p.apply_ninv(torch.zeros(40, dtype=f32)), TypeError),
        (lambda: p.scatter(torch.zeros(12, dtype=f64)), ValueError),
        (lambda: p.precond(torch.zeros(12, dtype=f32), mm.MM_PREC_BD, mm.MM_FP64), TypeError),
        (lambda: p.build_coarse(4, bprime=torch.zeros(12, dtype=f32)), TypeError),
        (lambda: p.grad(torch.zeros(40, dtype=f64), torch.zeros(12, dtype=f64), torch.zeros(11, dtype=f64)),
         ValueError),
        (lambda: p.apply_A_batch(torch.zeros(2, 12, dtype=f64)), TypeError),
        (lambda: p.apply_A_batch(torch.zeros(12, dtype=f32)), ValueError),      # 1-D: not [R, n]
        (lambda: p.solve_batch(torch.zeros(3, 41, dtype=f64)), ValueError),
        (lambda: p.solve(object()), TypeError),
    ]
    for call, exc in cases:
        with pytest.raises(exc, match="expected|unsupported array type"):
            call()


C_CONSUMER = r"""
#include <stdio.h>
#include <string.h>
#include "mm.h"

/* a plain C99 caller: every declared entry point is referenced (so the link resolves all
 * of them) and the calls that need no GPU are made */
typedef void (*any_fn)(void);
int main(void) {
    any_fn fns[] = {
%s
    };
    size_t i;
    mm_plan_t plan = NULL;
    mm_opts opts;
    for (i = 0; i < sizeof fns / sizeof fns[0]; ++i)
        if (fns[i] == NULL) return 3;
    memset(&opts, 0, sizeof opts);
    if (mm_plan(&plan, NULL, 0, 0, NULL, NULL, 0, NULL, NULL, 0, &opts) != MM_ERR_ARG || plan != NULL) return 4;
    if (mm_apply_A(NULL, MM_FP64, NULL, NULL) != MM_ERR_ARG) return 5;
    if (strstr(mm_version(), "sm_103a") == NULL) return 6;
    if (mm_launch_count() < 0) return 7;
    mm_destroy(NULL);
    printf("%%s\n", mm_version());
    return 0;
}
"""


def test_header_compiles_as_c_and_links(tmp_path):
    """include/mm.h is plain C (C99, pedantic) and a C program links every symbol it
    declares from libmm.so."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1408_3048_gb300 import build
    path = build.build()
    refs = "\n".join(f"        (any_fn){name}," for name in _declared())
    (tmp_path / "consumer.c").write_text(C_CONSUMER % refs)
    exe = tmp_path / "consumer"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-Wno-cast-function-type",
                    "-I", os.path.join(ROOT, "include"), str(tmp_path / "consumer.c"), path,
                    "-Wl,-rpath," + os.path.dirname(path), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert "sm_103a" in r.stdout


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding passes (mm_psd, mm_opts, mm_stats, mm_solve_opts) has the
    size and field offsets of include/mm.h as a C compiler lays it out."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1408_3048_gb300 import mm
    structs = {"mm_psd": mm.mm_psd, "mm_opts": mm.mm_opts, "mm_stats": mm.mm_stats,
               "mm_solve_opts": mm.mm_solve_opts}
    lines = []
    for cname, cls in structs.items():
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            cfield = "lambda" if fname == "lambda_" else fname
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {cfield}));')
    src = "#include <stddef.h>\n#include <stdio.h>\n#include \"mm.h\"\nint main(void) {\n" + "\n".join(lines) + \
          "\n    return 0;\n}\n"
    (tmp_path / "layout.c").write_text(src)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(tmp_path / "layout.c"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert c[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert c[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def _header_prototypes():
    """name -> (return type, [argument types]) for every function declared in mm.h."""
    with open(os.path.join(ROOT, "include", "mm.h")) as f:
        txt = re.sub(r"/\*.*?\*/", " ", f.read(), flags=re.S)
    protos = {}
    for m in re.finditer(r"^\s*((?:const\s+)?[a-z_0-9]+\s*\**)\s*(mm_[A-Za-z_0-9]+)\s*\(([^)]*)\)\s*;", txt,
                         re.M | re.S):
        ret, name, args = m.group(1), m.group(2), m.group(3)
        args = [" ".join(a.split()) for a in args.split(",")]
        protos[name] = (" ".join(ret.split()), [] if args == ["void"] else args)
    return protos


def _kind(c_decl):
    """Type class of a C parameter or return type: pointer, int32, int64, double, void."""
    if "*" in c_decl or c_decl.startswith("mm_plan_t"):
        return "ptr"
    t = c_decl.replace("const ", "").split()[0]
    return {"int32_t": "i32", "int": "i32", "mm_status": "i32", "int64_t": "i64", "double": "f64",
            "void": "void"}[t]


def _ctypes_kind(t):
    import ctypes as C
    if t is None:
        return "void"
    if t in (C.c_void_p, C.c_char_p) or issubclass(t, C._Pointer):
        return "ptr"
    return {C.c_int32: "i32", C.c_int: "i32", C.c_int64: "i64", C.c_double: "f64"}[t]


def test_binding_signatures_match_the_header_prototypes():
    from paper_1408_3048_gb300 import mm
    protos = _header_prototypes()
    assert sorted(protos) == _declared()
    for name, (ret, args) in protos.items():
        res, argt = mm._SIGS[name]
        assert _ctypes_kind(res) == _kind(ret), (name, "return")
        assert len(argt) == len(args), (name, len(argt), len(args))
        for i, (a, t) in enumerate(zip(args, argt)):
            assert _ctypes_kind(t) == _kind(a), (name, i, a)
