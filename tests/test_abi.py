"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/dd_nls.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "dd_nls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dd_(?:nls|cnn)_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1603_05110_gb300 import binding, build
    build.build()
    return binding.load()


def test_library_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 11
    for s in syms:
        assert hasattr(lib, s), s
    from paper_1603_05110_gb300 import binding
    assert set(syms) == set(binding.SYMBOLS)


def test_default_params_and_struct_layout(lib):
    from paper_1603_05110_gb300 import binding
    p = binding.default_params(nx=64, ny=40, n_strips=4)
    assert p.nx == 64 and p.n_strips == 4 and p.lap == 1.0 and p.tol == 1e-10
    assert p.gmres_restart == 30 and p.max_schwarz > 0


def test_ctypes_mirrors_match_the_c_layout(tmp_path):
    """Every field offset and struct size of the ctypes mirrors equals the C compiler's."""
    import shutil
    import subprocess
    from paper_1603_05110_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dd_nls.h"', "int main(void){"]
    expect = []
    for cname, cls in (("dd_nls_params", binding.Params), ("dd_nls_stats", binding.Stats),
                       ("dd_nls_profile", binding.Profile)):
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(cls))
        for f, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
            expect.append(getattr(cls, f).offset)
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == expect


def test_create_rejects_bad_sizes_without_touching_the_gpu(lib):
    import numpy as np
    from paper_1603_05110_gb300 import binding
    p = binding.default_params(nx=30, ny=8, n_strips=4)       # 30 % 4 != 0
    u0 = np.zeros((9, 31), np.complex128)
    with pytest.raises(binding.DDNLSError) as e:
        binding.Solver(p, u0)
    assert e.value.code == 1


BAD_PARAMS = {
    "nan_dt": dict(dt=float("nan")),
    "inf_kappa": dict(kappa=float("inf")),
    "nan_tol": dict(tol=float("nan")),
    "negative_tol": dict(nl_tol=-1e-12),
    "unknown_bc": dict(bc=7),
    "unknown_algorithm": dict(algorithm=5),
    "unknown_guess": dict(guess=3),
    "unknown_psolve": dict(psolve=4),
    "unknown_precision": dict(precision=9),
    "negative_nl_adapt": dict(nl_adapt=-0.1),
    "pade_order": dict(tc=1, pade_m=0),
    "robin_p": dict(p=0.0),
    "layout": dict(solver_layout=3),
}


@pytest.mark.parametrize("case", sorted(BAD_PARAMS))
def test_create_rejects_bad_parameters_without_touching_the_gpu(lib, case):
    """Every enum field one of its values, every real field finite and in range: EINVAL from
    dd_nls_create, from dd_nls_batch_create (naming the instance) and from the no-allocation
    step, all before any device work."""
    import numpy as np
    from paper_1603_05110_gb300 import binding
    kw = dict(nx=16, ny=8, n_strips=2, **BAD_PARAMS[case])
    u0 = np.zeros((9, 17), np.complex128)
    with pytest.raises(binding.DDNLSError) as e:
        binding.Solver(binding.default_params(**kw), u0)
    assert e.value.code == 1, str(e.value)
    with pytest.raises(binding.DDNLSError) as e:
        binding.Batch([dict(nx=16, ny=8, n_strips=2), kw], [u0, u0])
    assert e.value.code == 1 and "instance 1" in str(e.value), str(e.value)


def test_create_rejects_a_strip_beyond_32_bit_indexing(lib):
    import numpy as np
    from paper_1603_05110_gb300 import binding
    ny = 1 << 20                                                # ny + 1 nodes per column > 2^20
    with pytest.raises(binding.DDNLSError) as e:
        binding.Solver(binding.default_params(nx=1, ny=ny, n_strips=1), np.zeros((ny + 1, 2), np.complex128))
    assert e.value.code == 1 and "too large" in str(e.value)


@pytest.mark.parametrize("case", ["pade", "gmres", "dw_tight_tol", "mixed_precision", "trap", "mixed_inner_tol",
                                  "mixed_relax"])
def test_batch_create_rejects_unsupported_forms_without_touching_the_gpu(lib, case):
    """Batched instances take Robin transmission, the classical or the modal-preconditioned
    algorithm, one precision and one set of strip-solver settings for the whole batch, a static
    V, and nl_tol >= 1e-12 with the double-word residual; anything else is EINVAL before any
    device work."""
    import numpy as np
    from paper_1603_05110_gb300 import binding
    base = dict(nx=16, ny=8, n_strips=2, tol=1e-8, nl_tol=1e-11)
    prms = [dict(base), dict(base)]
    if case == "pade":
        prms[1].update(tc=binding.TC_PADE, pade_m=4)
    elif case == "gmres":
        prms[1].update(algorithm=binding.PRECONDITIONED, psolve=binding.PSOLVE_GMRES)
    elif case == "dw_tight_tol":
        for q in prms:
            q.update(precision=binding.FP32_DW, nl_tol=1e-13)
    elif case == "mixed_precision":
        prms[1].update(precision=binding.FP32_INNER)
    elif case == "trap":
        prms[1].update(trap_gx=1.0, trap_gy=1.2)
    elif case == "mixed_inner_tol":
        prms[1].update(inner_tol=1e-3)
    else:
        prms[1].update(nl_relax=0.5)
    u0 = [np.zeros((9, 17), np.complex128) for _ in prms]
    with pytest.raises(binding.DDNLSError) as e:
        binding.Batch(prms, u0)
    assert e.value.code == 1, str(e.value)


def test_cnn_create_rejects_an_image_beyond_32_bit_indexing(lib):
    out = ctypes.c_void_p()
    assert lib.dd_cnn_create(1 << 15, 1 << 14, None, ctypes.byref(out)) == 1
    assert not out.value
    assert b"2^28" in lib.dd_nls_last_error(None)
