"""Host-side checks of the C ABI that need no GPU.

The library must load, export every function include/tsdf.h declares, and
reject invalid arguments before touching the device.
"""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def T():
    from paper_1602_06645_gb300 import build as b
    b.build()
    import paper_1602_06645_gb300 as T
    T.load()
    return T


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tsdf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(tsdf_[a-z_]+)\s*\(", text))
    return sorted(n for n in names if n not in ("tsdf_status",))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("tsdf_create", "tsdf_integrate", "tsdf_read", "tsdf_destroy", "tsdf_save", "tsdf_load"):
        assert n in names


def test_library_exports_every_declared_symbol(T):
    lib = ctypes.CDLL(T.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(T.EXPORTS) == declared_functions()


def test_python_binding_has_the_c_names(T):
    for n in declared_functions():
        assert callable(getattr(T, n)), n


def test_status_strings(T):
    assert T.tsdf_status_string(0) == "ok"
    assert "invalid" in T.tsdf_status_string(-1)
    assert T.tsdf_status_string(12345) == "unknown status"


def test_params_default(T):
    p = T.tsdf_params_default()
    assert all(math.isnan(v) for v in p.origin)
    assert abs(p.sigma - 0.020) < 1e-9  # the paper's 20 mm (Eq. 7)
    assert math.isnan(p.band)
    assert p.culling == 1 and p.update_free_space == 1 and p.colour_mode == 0 and p.sample_mode == 0


@pytest.mark.parametrize("dims_geo,dims_col,vs,mu,mw", [
    ((0, 8, 8), (16, 16, 16), 0.01, 0.03, 64),        # dims <= 0
    ((8, 8, 8), (16, 16, 17), 0.01, 0.03, 64),        # anisotropic ratio
    ((8, 8, 8), (72, 72, 72), 0.01, 0.03, 64),        # colour/geometry ratio above 8
    ((8, 8, 5000), (8, 8, 5000), 0.01, 0.03, 64),     # dims > 4096
    ((8, 8, 8), (16, 16, 16), 0.0, 0.03, 64),         # voxel size <= 0
    ((8, 8, 8), (16, 16, 16), 0.01, -1.0, 64),        # mu <= 0
    ((8, 8, 8), (16, 16, 16), float("nan"), 0.03, 64),
    ((8, 8, 8), (16, 16, 16), 0.01, 0.03, 0),         # max_weight outside 1..255
    ((8, 8, 8), (16, 16, 16), 0.01, 0.03, 256),
])
def test_create_rejects_invalid_arguments(T, dims_geo, dims_col, vs, mu, mw):
    with pytest.raises(T.TsdfError) as e:
        T.tsdf_create(dims_geo, dims_col, vs, mu, mw)
    assert e.value.status == T.TSDF_ERR_INVALID_ARG


def test_create_rejects_bad_params(T):
    for field, value in (("sigma", 0.0), ("sigma", float("inf")), ("colour_mode", 2), ("sample_mode", -1),
                         ("band", -0.5)):
        p = T.tsdf_params_default()
        setattr(p, field, value)
        with pytest.raises(T.TsdfError) as e:
            T.tsdf_create_ex((8, 8, 8), (16, 16, 16), 0.01, 0.03, 64, p)
        assert e.value.status == T.TSDF_ERR_INVALID_ARG


def test_null_handle_calls_are_rejected(T):
    lib = T.load()
    assert lib.tsdf_integrate(None, None, T.tsdf_image_size(1, 1), None, T.tsdf_image_size(1, 1), None, None,
                              None, None) == T.TSDF_ERR_INVALID_ARG
    assert lib.tsdf_read(None, None, None, None) == T.TSDF_ERR_INVALID_ARG
    assert lib.tsdf_save(None, b"x") == T.TSDF_ERR_INVALID_ARG
    assert lib.tsdf_get_info(None, None) == T.TSDF_ERR_INVALID_ARG
    assert lib.tsdf_stats_request(None, 0) == T.TSDF_ERR_INVALID_ARG
    assert lib.tsdf_stats_collect(None, 0, None) == T.TSDF_ERR_INVALID_ARG
    lib.tsdf_destroy(None)  # ignored


def test_stats_copy_size_matches_the_header(T):
    text = open(os.path.join(ROOT, "include", "tsdf.h")).read()
    m = re.search(r"#define TSDF_STATS_COPY_BYTES (\d+)", text)
    assert m and int(m.group(1)) == T.STATS_COPY_BYTES
