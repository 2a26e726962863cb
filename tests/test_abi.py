"""CPU checks of the C ABI: the library builds, loads and exports every
function include/abm.h declares; host-side argument checks that run before
any CUDA call reject bad plans.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_1611_08678_gb300 import abm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(abm_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = abm.load()
    declared = _declared_functions()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(abm.EXPORTS) <= declared


def test_system_catalogue_dims():
    lib = abm.load()
    assert [lib.abm_system_dim(i) for i in range(7)] == [1, 1, 3, 3, 3, 3, 3]
    assert [lib.abm_system_nparams(i) for i in range(7)] == [3, 9, 3, 3, 3, 3, 8]
    assert lib.abm_system_dim(17) == -1
    assert lib.abm_system_dim(-1) == -1


def test_system_catalogue_agrees_with_the_oracle():
    """The library and the oracle number and size the right-hand sides alike
    (two catalogues written separately; the tests pass system names to both)."""
    import oracle
    lib = abm.load()
    assert set(abm.SYSTEMS) == set(oracle.SYSTEMS)
    for name, sid in abm.SYSTEMS.items():
        assert sid == oracle.SYSTEMS[name], name
        assert lib.abm_system_dim(sid) == oracle.dim(name), name
        assert lib.abm_system_nparams(sid) == oracle.nparams(name), name


def test_plan_create_rejects_bad_options_before_any_cuda_call():
    lib = abm.load()
    h = ctypes.c_void_p()
    o = abm.PlanOpts()
    lib.abm_plan_opts_default(ctypes.byref(o))
    o.n_max = 0
    assert lib.abm_plan_create(ctypes.byref(h), 2, ctypes.byref(o)) == 1
    o.n_max = 10
    o.reserved[3] = 1
    assert lib.abm_plan_create(ctypes.byref(h), 2, ctypes.byref(o)) == 1
    o.reserved[3] = 0
    o.max_batch = -1
    assert lib.abm_plan_create(ctypes.byref(h), 2, ctypes.byref(o)) == 1
    o.max_batch = 0
    assert lib.abm_plan_create(ctypes.byref(h), 99, ctypes.byref(o)) == 1
    o.tile_B = 48
    assert lib.abm_plan_create(ctypes.byref(h), 2, ctypes.byref(o)) == 6
    assert not h.value


@pytest.mark.parametrize("field,value,status", [
    ("prec", 4, 1), ("prec", -1, 1), ("near_warps", 4, 1), ("near_warps", 6, 1),
    ("far_split", -1, 1), ("far_split", 65, 1), ("near_split", 3, 1), ("near_split", 32, 1),
    ("far_ctas", -2, 1), ("spin_timeout_cycles", -5, 1), ("tile_B", -64, 1), ("tile_B", 128, 6),
    ("corrector_passes", -1, 1), ("corrector_passes", 9, 1),
])
def test_plan_options_outside_their_documented_sets_are_rejected(field, value, status):
    """Each option is checked against the values include/abm.h documents before
    the plan touches the device: nothing is allocated and no plan is returned."""
    lib = abm.load()
    h = ctypes.c_void_p()
    o = abm.PlanOpts()
    lib.abm_plan_opts_default(ctypes.byref(o))
    o.n_max = 16
    setattr(o, field, value)
    assert lib.abm_plan_create(ctypes.byref(h), 2, ctypes.byref(o)) == status
    assert not h.value


def test_tensor_core_precisions_need_three_components_and_64_row_tiles():
    lib = abm.load()
    h = ctypes.c_void_p()
    o = abm.PlanOpts()
    lib.abm_plan_opts_default(ctypes.byref(o))
    o.n_max = 16
    for prec in (2, 3):
        o.prec = prec
        o.tile_B = 0
        assert lib.abm_plan_create(ctypes.byref(h), abm.SYSTEMS["linear"], ctypes.byref(o)) == 6
        o.tile_B = 32
        assert lib.abm_plan_create(ctypes.byref(h), abm.SYSTEMS["lorenz"], ctypes.byref(o)) == 6
    assert not h.value


def test_product_path_has_no_oracle_or_cpu_fallback():
    """The package never imports the oracle, and the binding raises without a GPU."""
    pkg = os.path.join(ROOT, "paper_1611_08678_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "abm_oracle" not in text, fn
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError):
            abm.Plan("lorenz", n_max=10)


def test_checked_library_exports_the_same_symbols():
    """libabm_gb300_checked.so is the same sources compiled with ABM_CHECKED."""
    lib = abm.load(abm.CHECKED_LIB_PATH)
    declared = _declared_functions()
    assert not [n for n in sorted(declared) if not hasattr(lib, n)]


def test_only_the_checked_build_accepts_an_offset_index():
    """The testing option that moves one output row past the end of Y is
    refused by the plain library before any CUDA call: without the checks it
    would write outside the buffer."""
    lib = abm.load()
    h = ctypes.c_void_p()
    o = abm.PlanOpts()
    lib.abm_plan_opts_default(ctypes.byref(o))
    o.n_max, o.max_batch, o.test_bad_index = 100, 4, 1
    assert lib.abm_plan_create(ctypes.byref(h), 2, ctypes.byref(o)) == 6
    assert not h.value
    o.test_bad_index = -1
    assert lib.abm_plan_create(ctypes.byref(h), 2, ctypes.byref(o)) == 1
