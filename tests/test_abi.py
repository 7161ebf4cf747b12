"""CPU-side checks of the C ABI: the library builds and loads, exports every
entry point that include/nnp.h declares, and its struct layout matches what
a C compiler makes of the header.  No call here needs a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nnp.h")


@pytest.fixture(scope="module")
def L():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    return P.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nnp_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    import paper_2604_21441_b300 as P
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(P.ABI_FUNCTIONS)
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (nnp_\w+)", out))
    assert set(names) <= exported


def test_config_layout_matches_header(tmp_path):
    import paper_2604_21441_b300 as P
    fields = [f[0] for f in P.Config._fields_]
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"nnp.h\"\nint main(void){\n"
    prog += 'printf("%zu\\n", sizeof(nnp_config));\n'
    for f in fields:
        prog += f'printf("%zu\\n", offsetof(nnp_config, {f}));\n'
    prog += "return 0;}\n"
    c = tmp_path / "layout.c"
    c.write_text(prog)
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    vals = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert vals[0] == ctypes.sizeof(P.Config)
    for f, off in zip(fields, vals[1:]):
        assert getattr(P.Config, f).offset == off, f


def test_config_init_defaults(L):
    import paper_2604_21441_b300 as P
    cfg = P.Config()
    zs = (ctypes.c_int32 * 8)(1, 6, 7, 8)
    assert L.nnp_config_init(ctypes.byref(cfg), 4, zs) == 0
    assert cfg.n_species == 4 and list(cfg.atomic_numbers)[:4] == [1, 6, 7, 8]
    assert (cfg.rc_r, cfg.eta_r, cfg.rc_a, cfg.eta_a, cfg.zeta) == (5.2, 16.0, 3.5, 8.0, 32.0)
    assert abs(cfg.shf_r[15] - 4.93125) < 1e-12 and abs(cfg.shf_a[3] - 2.85) < 1e-12
    assert list(cfg.hidden) == [160, 128, 96] and cfg.celu_alpha == 0.1
    # invalid: not ascending, too many species, null
    bad = (ctypes.c_int32 * 8)(8, 1)
    assert L.nnp_config_init(ctypes.byref(cfg), 2, bad) == 1
    assert L.nnp_config_init(ctypes.byref(cfg), 9, zs) == 1
    assert L.nnp_config_init(None, 2, zs) == 1


def test_create_rejects_bad_configs_before_touching_the_gpu(L):
    import paper_2604_21441_b300 as P
    zs = (ctypes.c_int32 * 8)(1, 8)
    h = ctypes.c_void_p()
    for field, value, code in [("zeta", 3.0, 3), ("n_rad", 8, 3), ("precision", 7, 1),
                               ("celu_alpha", 0.0, 1)]:
        cfg = P.Config()
        L.nnp_config_init(ctypes.byref(cfg), 2, zs)
        setattr(cfg, field, value)
        assert L.nnp_create(ctypes.byref(cfg), ctypes.byref(h)) == code, field
        assert h.value is None
        assert len(L.nnp_last_error(None)) > 0
    cfg = P.Config()
    L.nnp_config_init(ctypes.byref(cfg), 2, zs)
    cfg.hidden[0] = 128
    assert L.nnp_create(ctypes.byref(cfg), ctypes.byref(h)) == 3


def test_param_count_formula():
    # S * (D*160 + 160 + 160*128 + 128 + 128*96 + 96 + 96 + 1)
    for S, D in ((2, 128), (4, 384)):
        assert S * (D * 160 + 160 + 160 * 128 + 128 + 128 * 96 + 96 + 96 + 1) > 0


def test_no_oracle_in_product_path():
    """The package never imports, links or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_2604_21441_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "nnp_oracle" not in txt and "liboracle" not in txt, f
