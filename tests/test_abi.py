"""The C-ABI library loads and exports every entry point declared in
include/pairdiag.h (no GPU needed: no compute calls are made)."""
import ctypes
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
HEADER = ROOT / "include" / "pairdiag.h"


def declared_symbols():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pairdiag_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2001_01978_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pairdiag_create", "pairdiag_ground_state", "pairdiag_hx_dev", "pairdiag_destroy",
                     "pairdiag_basis_dev", "pairdiag_rank_dev"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(str(libpath))
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", str(libpath)], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pairdiag_[a-z0-9_]+)", out))
    assert set(declared_symbols()) <= exported


def test_binding_covers_the_header(libpath):
    import paper_2001_01978_gb300 as pd
    assert set(declared_symbols()) == set(pd.exported_symbols())


def test_host_only_entry_points(libpath):
    """Entry points that need no device: defaults and status strings."""
    import paper_2001_01978_gb300 as pd
    o = pd.pairdiag_default_options()
    assert o.window == 20 and o.precision == pd.PD_PREC_FP64 and o.mode == 0
    assert pd.pairdiag_strerror(pd.PD_ENOCONV) == "Lanczos did not converge"
    assert pd.pairdiag_strerror(pd.PD_OK) == "success"


def test_no_cpu_fallback_in_product_path():
    """The package never imports the oracle (the product path fails loudly instead)."""
    pkg = ROOT / "paper_2001_01978_gb300"
    for f in pkg.rglob("*.py"):
        src = f.read_text()
        assert "import oracle" not in src and "from oracle" not in src, f


def test_tune_table_host_only(libpath):
    import paper_2001_01978_gb300 as pd
    assert pd.pairdiag_tune_get(20, 10, 1) == (0, 0)
    pd.pairdiag_tune_set(20, 10, 1, 11, 2)
    assert pd.pairdiag_tune_get(20, 10, 1) == (11, 2)
    pd.pairdiag_tune_set(20, 10, 1, 0, 0)
    assert pd.pairdiag_tune_get(20, 10, 1) == (0, 0)
    with pytest.raises(pd.PairDiagError):
        pd.pairdiag_tune_set(20, 10, 1, 14, 1)


def test_odd_ground_state_argument_errors(libpath):
    """Argument checks of the odd-mass entry point return PD_EINVAL before any
    device call."""
    import numpy as np
    import paper_2001_01978_gb300 as pd
    e = np.arange(6.0)
    G = np.full((6, 6), -0.3)
    bad = [
        dict(omega=1, n_pairs=0, e=e[:1], G=G[:1, :1]),        # no orbit left to pair in
        dict(omega=6, n_pairs=6, e=e, G=G),                    # 13 particles in 6 orbits
        dict(omega=6, n_pairs=-1, e=e, G=G),
        dict(omega=6, n_pairs=2, e=e, G=G, block=6),
        dict(omega=6, n_pairs=2, e=e, G=G, block=-2),
        dict(omega=6, n_pairs=2, e=e, G=G, tol=-1.0),
        dict(omega=6, n_pairs=2, e=e, G=G + np.triu(np.full((6, 6), 1e-3), 1)),
        dict(omega=6, n_pairs=2, e=np.r_[e[:5], np.nan], G=G),
        dict(omega=6, n_pairs=2, e=e, G=G, opt=pd.pairdiag_default_options(start=pd.PD_START_USER)),
        dict(omega=6, n_pairs=2, e=e, G=G, opt=pd.pairdiag_default_options(start=pd.PD_START_MLP)),
    ]
    for kw in bad:
        kw.setdefault("tol", 1e-10)
        with pytest.raises(pd.PairDiagError) as err:
            pd.pairdiag_odd_ground_state(**kw)
        assert err.value.code == pd.PD_EINVAL, kw


def test_binding_shape_checks_need_no_device(libpath):
    """The binding rejects mis-shaped host inputs before calling the library."""
    import numpy as np
    import paper_2001_01978_gb300 as pd
    with pytest.raises(ValueError):
        pd.pairdiag_odd_ground_state(6, 2, np.zeros(5), np.zeros((6, 6)), 1e-10)
    with pytest.raises(ValueError):
        pd.pairdiag_odd_ground_state(6, 2, np.zeros(6), np.zeros((6, 5)), 1e-10)
    with pytest.raises(ValueError):
        pd.pairdiag_create(6, 2, np.zeros(6), np.zeros((5, 5)))


def test_multidot_wrappers_check_sizes_before_any_call():
    """The library cannot see buffer sizes, so the binding rejects a short out,
    Q or p and any dtype other than float32/float64 before a pointer is passed
    (CPU tensors: nothing reaches the library or a GPU)."""
    torch = pytest.importorskip("torch")
    import paper_2001_01978_gb300 as pd
    Q = torch.zeros(3, 8, dtype=torch.float64)
    p = torch.zeros(8, dtype=torch.float64)
    with pytest.raises(ValueError, match="out has 2 elements"):
        pd.pairdiag_multidot_noalloc(Q, 8, 3, p, 8, torch.zeros(2, dtype=torch.float64))
    with pytest.raises(ValueError, match="Q has 24 elements"):
        pd.pairdiag_multidot_noalloc(Q, 9, 3, p, 8, torch.zeros(3, dtype=torch.float64))
    with pytest.raises(ValueError, match="p has 7 elements"):
        pd.pairdiag_multidot_noalloc(Q, 8, 3, p[:7], 8, torch.zeros(3, dtype=torch.float64))
    with pytest.raises(TypeError, match="float64 or float32"):
        pd.pairdiag_multidot_noalloc(Q.to(torch.float16), 8, 3, p.to(torch.float16), 8,
                                     torch.zeros(3, dtype=torch.float64))
    with pytest.raises(TypeError, match="out must be float64"):
        pd.pairdiag_multidot_noalloc(Q, 8, 3, p, 8, torch.zeros(3, dtype=torch.float32))
    with pytest.raises(ValueError, match="Q has 24 elements"):
        pd.pairdiag_multidot(None, Q, 8, 4, p, 8)
    # sizes that fit pass the checks and stop at the device check
    with pytest.raises(TypeError, match="CUDA tensor"):
        pd.pairdiag_multidot_noalloc(Q, 8, 3, p, 8, torch.zeros(3, dtype=torch.float64))


def test_host_array_wrappers_check_shapes_before_any_call(libpath):
    """The library reads rows * 16 feature floats, num_params parameters, omega
    weights per handle, omega and omega^2 inputs per batch problem and m - 1
    off-diagonal entries from host pointers it cannot size, so the binding
    rejects any other shape before a pointer is passed (a null network or
    handle: nothing reaches a device)."""
    import numpy as np
    import paper_2001_01978_gb300 as pd
    assert pd.pairdiag_omega(None) == -1
    with pytest.raises(ValueError, match="theta must hold"):
        pd.pairdiag_mlp_set_params(None, np.zeros(pd.pairdiag_mlp_num_params() - 1))
    with pytest.raises(ValueError, match=r"\[rows, 16\]"):
        pd.pairdiag_mlp_forward(None, np.zeros((5, 15)))
    with pytest.raises(ValueError, match=r"\[rows, 16\]"):
        pd.pairdiag_mlp_forward(None, np.zeros(16))
    with pytest.raises(ValueError, match=r"target must be \[5\]"):
        pd.pairdiag_mlp_loss_grad(None, np.zeros((5, 16)), np.zeros(4))
    with pytest.raises(ValueError, match=r"target must be \[5\]"):
        pd.pairdiag_mlp_train(None, np.zeros((5, 16)), np.zeros((5, 1)), 3)
    with pytest.raises(ValueError, match="steps"):
        pd.pairdiag_mlp_train(None, np.zeros((5, 16)), np.zeros(5), -1)
    with pytest.raises(ValueError, match="not a valid handle"):
        pd.pairdiag_set_start_weights(None, np.zeros(6))
    with pytest.raises(ValueError, match="problem 1"):
        pd.pairdiag_batch_ground_state([(6, 2, np.zeros(6), np.zeros((6, 6))),
                                        (7, 3, np.zeros(7), np.zeros((6, 6)))], 1e-8)
    with pytest.raises(ValueError, match="at least one problem"):
        pd.pairdiag_batch_ground_state([], 1e-8)
    with pytest.raises(ValueError, match="off-diagonal"):
        pd.pairdiag_tridiag_lowest(None, np.zeros(4), np.zeros(2))


def test_create_and_batch_reject_invalid_input_before_any_device_call(libpath):
    """Host-side fault injection: out-of-range sizes, non-finite or asymmetric
    inputs and bad options make pairdiag_create and the batch return PD_EINVAL
    (or PD_ENOTSUP for a form the batch does not run) before any CUDA call, so
    these run on a machine without a GPU."""
    import numpy as np
    import paper_2001_01978_gb300 as pd
    e = np.arange(6.0)
    G = np.full((6, 6), -0.3)
    asym = G + np.triu(np.full((6, 6), 1e-3), 1)
    Gnan = G.copy()
    Gnan[2, 3] = Gnan[3, 2] = np.nan
    Ginf = G.copy()
    Ginf[1, 1] = np.inf
    opt = pd.pairdiag_default_options
    bad_create = [
        (6, 7, e, G, None),                      # more pairs than orbits
        (6, -1, e, G, None),
        (6, 2, e, asym, None),                   # G must be symmetric (reading r4)
        (6, 2, np.r_[e[:5], np.nan], G, None),
        (6, 2, e, Gnan, None),
        (6, 2, e, Ginf, None),
        (6, 2, e, G, opt(window=0)),
        (6, 2, e, G, opt(window=65)),
        (6, 2, e, G, opt(precision=2)),
        (6, 2, e, G, opt(mode=2)),
        (6, 2, e, G, opt(low_bits=40)),
        (6, 2, e, G, opt(max_restarts=-1)),
        (6, 2, e, G, opt(hx_variant=6)),
        (6, 2, e, G, opt(start=5)),
    ]
    for om, n, ee, GG, o in bad_create:
        with pytest.raises(pd.PairDiagError) as err:
            pd.pairdiag_create(om, n, ee, GG, o)
        assert err.value.code == pd.PD_EINVAL, (om, n, o)
    ok = (6, 2, e, G)
    bad_batch = [
        ([ok, (6, 2, e, asym)], None, 1e-8, pd.PD_EINVAL),
        ([ok, (6, 2, np.r_[e[:5], np.inf], G)], None, 1e-8, pd.PD_EINVAL),
        ([ok, (6, 7, e, G)], None, 1e-8, pd.PD_EINVAL),
        ([ok], None, -1.0, pd.PD_EINVAL),
        ([ok], opt(window=0), 1e-8, pd.PD_EINVAL),
        ([ok], opt(precision=2), 1e-8, pd.PD_EINVAL),
        ([ok], opt(start=pd.PD_START_MLP), 1e-8, pd.PD_EINVAL),      # the learned start needs a network
        ([ok], opt(start=pd.PD_START_FIRST), 1e-8, pd.PD_ENOTSUP),
        ([ok], opt(mode=1), 1e-8, pd.PD_ENOTSUP),
    ]
    for probs, o, tol, code in bad_batch:
        with pytest.raises(pd.PairDiagError) as err:
            pd.pairdiag_batch_ground_state(probs, tol, o)
        assert err.value.code == code, (o, tol, err.value.code)
