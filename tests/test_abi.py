"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/ffmin.h declares (no compute call is made here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(ffmin_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_1810_03358_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("ffmin_create", "ffmin_destroy", "ffmin_energy", "ffmin_energy_grad",
                     "ffmin_minimize", "ffmin_options_default", "ffmin_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_and_binds_without_gpu(built):
    from paper_1810_03358_gb300 import ffmin
    L = ffmin.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    o = ffmin.ffmin_options_default()
    assert o.method == ffmin.FFMIN_LBFGS and o.lbfgs_m == 10 and o.gtol_inf == 0.1
    assert o.h0 == 0.1 and o.k_plus == 2.0 and o.k_minus == 0.5 and o.ls_par_K == 2
    assert L.ffmin_status_string(ffmin.FFMIN_ERR_LINESEARCH) == b"line search failed"


def test_binding_names_match_header():
    from paper_1810_03358_gb300 import ffmin
    assert set(ffmin.EXPORTS) == declared_functions()
    for name in ffmin.EXPORTS:
        assert callable(getattr(ffmin, name)), name


def test_create_rejects_bad_topology_on_host(built):
    # argument checks run before any CUDA call, so they work without a GPU
    import ctypes as C
    from types import SimpleNamespace
    import numpy as np
    from paper_1810_03358_gb300 import ffmin
    s = SimpleNamespace(charge=np.zeros(3), sigma=np.ones(3), epsilon=np.ones(3) * 0.1,
                        bond_idx=np.array([[0, 5]]), bond_k=np.ones(1), bond_r0=np.ones(1),
                        angle_idx=np.zeros((0, 3)), angle_k=np.zeros(0), angle_theta0=np.zeros(0),
                        dihedral_idx=np.zeros((0, 4)), dihedral_v=np.zeros((0, 4)), coulomb_c=0.0)
    keep = []
    top = ffmin._topology(s, keep)
    h = C.c_void_p()
    st = ffmin.lib().ffmin_create(C.byref(top), 1, 0, None, C.byref(h))
    assert st == ffmin.FFMIN_ERR_INVALID_ARG
    assert b"out of range" in ffmin.lib().ffmin_last_error(None)
    st = ffmin.lib().ffmin_create(C.byref(top), 0, 0, None, C.byref(h))
    assert st == ffmin.FFMIN_ERR_INVALID_ARG


def test_option_defaults_agree_with_the_oracle(built, oracle_mod):
    # the library's and the oracle's defaults are the readings of the paper
    # (first step 0.1 A, k+ = 2, k- = 0.5, eps_h = 1e-10, LS_PAR K = 2 with
    # G0, m = 10, |grad|_inf < 0.1); both sides set them independently
    from paper_1810_03358_gb300 import ffmin
    g = ffmin.ffmin_options_default()
    o, _ = oracle_mod.options()
    for k in ("method", "cg_variant", "ls", "lbfgs_m", "gtol_inf", "max_iter", "max_evals", "h0", "k_plus",
              "k_minus", "eps_h", "ls_par_K", "ls_par_g0", "gradfree_delta", "gradfree_parts", "fgm_restart"):
        assert getattr(g, k) == getattr(o, k), k
    assert (g.h0, g.k_plus, g.k_minus, g.ls_par_K, g.lbfgs_m, g.gtol_inf) == (0.1, 2.0, 0.5, 2, 10, 0.1)
    assert g.fgm_restart == 0  # Algorithm 1 as printed
