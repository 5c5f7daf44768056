"""The C ABI: the library builds, loads and exports every declared symbol;
argument errors are reported without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fvn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fvn_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def binding():
    import __graft_entry__ as ge
    ge.build()
    from paper_2209_09965_gb300 import fvn
    return fvn


def test_every_declared_symbol_is_exported(binding):
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(binding.lib, n), n
    assert set(names) == set(binding.EXPORTS)


def test_weight_count_matches_layer_table(binding):
    from paper_2209_09965_gb300 import workloads as wl
    assert binding.weight_count() == wl.net_param_count()
    assert binding.weight_count_recurrent() == wl.net_param_count(wl.NET_LAYERS_RECURRENT)
    assert wl.recurrent_weights(wl.net_weights(3)).size == binding.weight_count_recurrent()


def test_null_context_is_an_argument_error(binding):
    lib = binding.lib
    assert lib.fvn_make_mask(None, None, 4, 4, None, None, None, None) == -1
    assert lib.fvn_march(None, None, None, None, None, None, None, None, None, None) == -1
    assert lib.fvn_reconstruct(None, None, 4, 4, 0, None, None) == -1
    assert lib.fvn_render(None, None, None, None, None, None, 0, None, None, None) == -1
    assert lib.fvn_load_weights(None, None, 0) == -1
    assert b"ctx is NULL" in lib.fvn_last_error(None)
    assert lib.fvn_create(None) == -1


def test_training_entry_points_validate_before_launch(binding):
    lib = binding.lib
    assert lib.fvn_conv_fwd(None, 1, None, 0, 1, 4, 4, None, None, 1, 3, 1, None, None) == -1
    assert lib.fvn_conv_bwd(None, 1, None, 0, 1, 4, 4, None, 1, 3, None, None, None, None, None, None, None) == -1
    assert lib.fvn_avgpool2_fwd(None, 1, 3, 4, None, None) == -1
    assert lib.fvn_upsample2_bwd(None, 1, 4, 4, None, None) == -1
    assert lib.fvn_kp_blend_fwd(None, None, 1, 4, 4, None, None) == -1
    assert lib.fvn_loss_l1grad(None, None, 1, 4, 4, ctypes.c_float(1.0), None, None, None) == -1
    assert lib.fvn_adam_step(None, None, None, None, 0, 1, ctypes.c_float(1e-3), ctypes.c_float(0.9),
                             ctypes.c_float(0.999), ctypes.c_float(1e-8), None) == -1
    assert b"bad" in lib.fvn_last_error(None) or b"null" in lib.fvn_last_error(None)


def test_two_stage_weight_count_and_argument_checks(binding):
    from oracle import wnet as W
    from paper_2209_09965_gb300 import workloads as wl
    for cfg in (wl.WNET_PAPER, wl.WNET_SLIM, ((3, 5), 6, (4, 5)), ((8,), 4, (6,)), ((4, 5, 6, 7), 9, (3, 4, 5, 6))):
        assert binding.wnet_weight_count(cfg) == W.param_count(cfg) == wl.net_param_count(wl.wnet_layers(cfg))
    assert binding.wnet_weight_count(wl.WNET_PAPER) == 862741
    for bad in (((), 4, ()), ((4,) * 5, 4, (4,) * 5), ((0, 4), 4, (4, 4)), ((4, 4), 257, (4, 4))):
        c = binding.WnetConfigC()
        c.levels = len(bad[0])
        for s in range(min(len(bad[0]), 4)):
            c.enc[s], c.dec[s] = bad[0][s], bad[2][s]
        c.bot = bad[1]
        assert binding.lib.fvn_wnet_weight_count(ctypes.byref(c)) == 0
    assert binding.wnet_weight_count(((4,) * 5, 4, (4,) * 5)) == 0    # too deep: marshalled, then rejected
    lib = binding.lib
    assert lib.fvn_load_wnet_weights(None, None, None, 0) == -1
    assert lib.fvn_reconstruct_wnet(None, None, 4, 4, None, None) == -1
    assert lib.fvn_filter3_fwd(None, None, 1, 4, 4, None, None) == -1
    assert lib.fvn_filter3_bwd(None, None, 1, 4, 4, None, None, None, None) == -1
    assert lib.fvn_wnet_join_fwd(None, None, None, 1, 4, 4, None, None) == -1
    p = ctypes.c_void_p(16)   # never dereferenced: the odd size is rejected first
    assert lib.fvn_wnet_join_fwd(p, p, p, 1, 5, 4, p, None) == -1
    assert lib.fvn_wnet_join_bwd(p, p, p, 1, 4, 3, p, p, p, p, None) == -1
