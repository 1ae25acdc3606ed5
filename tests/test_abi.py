"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/ia.h declares, and rejects invalid configurations with
IA_ERR_ARG before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ia_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def ia():
    import paper_2212_10550_b300 as ia
    from paper_2212_10550_b300 import build
    build.build()
    ia.lib()
    return ia


def test_every_declared_symbol_is_exported(ia):
    names = _declared()
    assert {"ia_create", "ia_render", "ia_set_pose", "ia_update_occupancy", "ia_set_skeleton"} <= names
    for n in sorted(names):
        assert hasattr(ia.lib(), n), n


def test_version(ia):
    assert "sm_103a" in ia.ia_version()


def _cfg(ia, **kw):
    base = dict(n_levels=8, log2_table=14, level_res=[16, 24, 36, 54, 81, 121, 182, 273], max_samples=32,
                occ_res=32)
    base.update(kw)
    return ia.make_config(**base)


@pytest.mark.parametrize("bad", [dict(n_levels=0), dict(n_levels=17), dict(n_features=4), dict(log2_table=30),
                                 dict(mlp_width=32), dict(max_samples=0), dict(broyden_max_iter=0),
                                 dict(broyden_tol=0.0), dict(occ_res=1), dict(occ_dilate=9),
                                 dict(early_stop_T=2.0), dict(precision=7),
                                 dict(level_res=[1, 24, 36, 54, 81, 121, 182, 273])])
def test_invalid_config_is_rejected_on_the_host(ia, bad):
    with pytest.raises(ia.IAError) as e:
        ia.ia_create(_cfg(ia, **bad))
    assert e.value.status == ia.IA_ERR_ARG
    assert ia.ia_last_error(None)


def test_null_arguments(ia):
    ctx = C.c_void_p()
    assert ia.lib().ia_create(None, C.byref(ctx)) == ia.IA_ERR_ARG
    assert ia.lib().ia_render(None, 0, None, None, None, None, None) == ia.IA_ERR_ARG
    assert ia.lib().ia_set_pose(None, 1, None, None, None) == ia.IA_ERR_ARG
    ia.lib().ia_destroy(None)  # allowed


def test_null_context_of_the_training_split_and_pipeline_settings(ia):
    L = ia.lib()
    assert L.ia_train_forward(None, None, 0, None, None, None, None, None) == ia.IA_ERR_ARG
    assert L.ia_train_backward(None, None, None, None, None) == ia.IA_ERR_ARG
    assert L.ia_set_wait_limit(None, 0) == ia.IA_ERR_ARG
    assert L.ia_set_fault_injection(None, 0) == ia.IA_ERR_ARG
    assert L.ia_set_render_path(None, 0) == ia.IA_ERR_ARG
    assert L.ia_gather_probe(None, 1, 48, 1, 1, None, None) == ia.IA_ERR_ARG
    assert L.ia_atomic_probe(None, 1, 8, 1, 1, None) == ia.IA_ERR_ARG


def test_launch_tracing_state_machine(ia):
    """ia_profile_begin / ia_profile_end need no device when nothing launched:
    an empty profile, and the order errors."""
    with pytest.raises(ia.IAError) as e:
        ia.ia_profile_end()
    assert e.value.status == ia.IA_ERR_STATE
    ia.ia_profile_begin()
    with pytest.raises(ia.IAError) as e:
        ia.ia_profile_begin()
    assert e.value.status == ia.IA_ERR_STATE
    assert ia.ia_profile_end() == {}
    n = C.c_int(-1)
    assert ia.lib().ia_profile_begin() == ia.IA_OK
    assert ia.lib().ia_profile_end(None, -1, C.byref(n)) == ia.IA_ERR_ARG  # bad arguments: still open
    assert ia.lib().ia_profile_end(None, 0, C.byref(n)) == ia.IA_OK and n.value == 0
    assert ia.lib().ia_profile_end(None, 0, C.byref(n)) == ia.IA_ERR_STATE
