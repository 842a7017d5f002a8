"""The C ABI library loads, exports every function include/dsmc.h declares, and validates
arguments on the host (no GPU needed: these calls launch nothing)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2202_02264_gb300 import build
    build.build()
    return C.CDLL(build.LIB)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dsmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dsmc_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_symbol():
    from paper_2202_02264_gb300 import dsmc
    assert sorted(dsmc.EXPORTS) == declared_functions()


def _structs():
    from paper_2202_02264_gb300 import dsmc, workloads as W
    m = W.lgssm_d8()
    hm = dsmc.HostModel(m)
    return dsmc, W, hm


def test_sizes_and_argument_checks(lib):
    dsmc, W, hm = _structs()
    cfg = dsmc.make_config(1024, 1024, 7)
    s = dsmc.dsmc_state_sizes(cfg, hm)
    assert s == [1024 * 1024 * 8 * 4, 1024 * 1024 * 4, 1024 * 8, 1023 * 2 * 1024 * 4]
    ws = dsmc.dsmc_workspace_size(cfg, hm)
    assert ws > 0 and ws % 256 == 0
    for bad in [dict(K=0), dict(N=0), dict(N=20000)]:
        c = dsmc.make_config(bad.get("K", 8), bad.get("N", 8), 1)
        with pytest.raises(dsmc.DsmcError) as e:
            dsmc.dsmc_workspace_size(c, hm)
        assert e.value.code in (1, 2)
    # RS lifts the dense N limit
    c = dsmc.make_config(8, 20000, 1, resampler=dsmc.RS)
    assert dsmc.dsmc_workspace_size(c, hm) > 0
    # tensor-core precisions: BF16 for every dx, TF32 up to dx = 16, N <= 4096 when dense
    assert dsmc.dsmc_workspace_size(dsmc.make_config(8, 64, 1, compute=dsmc.BF16), hm) > 0
    assert dsmc.dsmc_workspace_size(dsmc.make_config(8, 64, 1, compute=dsmc.TF32), hm) > 0
    with pytest.raises(dsmc.DsmcError) as e:
        dsmc.dsmc_workspace_size(dsmc.make_config(8, 8192, 1, compute=dsmc.BF16), hm)
    assert e.value.code == 2
    hm16, hm32 = dsmc.HostModel(W.lgssm_dn(16)), dsmc.HostModel(W.lgssm_dn(32))
    assert dsmc.dsmc_workspace_size(dsmc.make_config(8, 64, 1, compute=dsmc.TF32), hm16) > 0
    assert dsmc.dsmc_workspace_size(dsmc.make_config(8, 64, 1, compute=dsmc.BF16), hm32) > 0
    with pytest.raises(dsmc.DsmcError) as e:
        dsmc.dsmc_workspace_size(dsmc.make_config(8, 64, 1, compute=dsmc.TF32), hm32)
    assert e.value.code == 2


def test_lazy_samplers_plan_no_dense_buffers(lib):
    """The lazy samplers (DSMC_RS, DSMC_RS_FACTORED, DSMC_MH) lift the dense N limit and plan
    neither tile sums nor tensor-core operands, whatever the precision field says; the
    systematic sampler is dense (same limit and buffers as multinomial); an unknown sampler
    is refused."""
    dsmc, W, hm = _structs()
    dense = dsmc.dsmc_workspace_size(dsmc.make_config(64, 1024, 1, compute=dsmc.BF16), hm)
    assert dsmc.dsmc_workspace_size(dsmc.make_config(64, 1024, 1, compute=dsmc.BF16,
                                                     resampler=dsmc.SYSTEMATIC), hm) == dense
    with pytest.raises(dsmc.DsmcError) as e:
        dsmc.dsmc_workspace_size(dsmc.make_config(8, 20000, 1, resampler=dsmc.SYSTEMATIC), hm)
    assert e.value.code == 2
    for res in (dsmc.RS, dsmc.RS_FACTORED, dsmc.MH):
        lazy_bf16 = dsmc.dsmc_workspace_size(dsmc.make_config(64, 1024, 1, resampler=res, compute=dsmc.BF16), hm)
        lazy_fp32 = dsmc.dsmc_workspace_size(dsmc.make_config(64, 1024, 1, resampler=res), hm)
        assert lazy_bf16 == lazy_fp32 < dense
        assert dsmc.dsmc_workspace_size(dsmc.make_config(8, 20000, 1, resampler=res), hm) > 0
    with pytest.raises(dsmc.DsmcError) as e:
        dsmc.dsmc_workspace_size(dsmc.make_config(8, 64, 1, resampler=5), hm)
    assert e.value.code == 1


def test_invalid_model_rejected(lib):
    dsmc, W, _ = _structs()
    m = W.sv(8)
    m.phi = 1.5
    hm = dsmc.HostModel(m)
    with pytest.raises(dsmc.DsmcError) as e:
        dsmc.dsmc_workspace_size(dsmc.make_config(8, 8, 1), hm)
    assert e.value.code == 1


def test_status_strings(lib):
    lib.dsmc_status_string.restype = C.c_char_p
    for code in [0, 1, 2, 3, 5, 6, 7, 8, 9, 10]:
        assert lib.dsmc_status_string(code)


def test_tile_cols_is_validated(lib):
    dsmc, W, _ = _structs()
    hm = dsmc.HostModel(W.lgssm_d4())
    ok = dsmc.make_config(8, 512, 1, tile_cols=64)
    assert dsmc.dsmc_workspace_size(ok, hm) > 0
    for bad, code in (((8, 512, 48), 1), ((8, 8192, 64), 2), ((8, 4096, 32), 2)):
        K, N, t = bad
        c = dsmc.make_config(K, N, 1, tile_cols=t)
        with pytest.raises(dsmc.DsmcError) as e:
            dsmc.dsmc_workspace_size(c, hm)
        assert e.value.code == code
