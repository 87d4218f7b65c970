"""Host-side logic of the C ABI that needs no GPU: the layout of mfp_desc as
the binding declares it (filled by the library's own mfp_desc_default) and
the argument checks of mfp_create, which run before any CUDA call."""
import ctypes

import pytest

from paper_1611_03029_gb300 import build


@pytest.fixture(scope="module")
def mfp():
    build.build()
    from paper_1611_03029_gb300 import mfpoisson
    return mfpoisson


def default_desc(mfp):
    d = mfp.MfpDesc()
    ctypes.memset(ctypes.byref(d), 0x7f, ctypes.sizeof(d))
    mfp.lib().mfp_desc_default(ctypes.byref(d))
    return d


def test_desc_defaults_land_in_their_fields(mfp):
    # a field the binding places at the wrong offset reads garbage here
    d = default_desc(mfp)
    assert (d.nx, d.ny, d.nz, d.degree) == (1, 1, 1, 1)
    assert (d.disc, d.n_levels, d.mapping) == (mfp.MFP_CG, 0, 0)
    assert (d.map_param, d.kappa, d.penalty_factor) == (0.0, 1.0, 1.0)
    assert (d.mg_precision, d.cheb_degree, d.eig_cg_iters) == (0, 5, 15)
    assert d.fp64_arith == mfp.MFP_ARITH_DF
    assert d.neumann_sides == 0
    assert (d.box_lo, d.box_hi) == (0.0, 1.0)
    assert not d.map_nodes


@pytest.mark.parametrize("field,value,msg", [
    ("neumann_sides", 63, "Dirichlet"),
    ("neumann_sides", -1, "neumann_sides"),
    ("neumann_sides", 64, "neumann_sides"),
    ("box_hi", 0.0, "box"),
    ("box_lo", float("nan"), "box"),
    ("degree", 9, "degree"),
    ("kappa", 0.0, "kappa")])
def test_create_rejects_bad_descriptions(mfp, field, value, msg):
    d = default_desc(mfp)
    setattr(d, field, value)
    h = ctypes.c_void_p()
    st = mfp.lib().mfp_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == mfp.MFP_ERR_ARG
    assert not h.value
    assert msg in mfp.lib().mfp_last_error().decode()


def test_create_rejects_node_mapping_without_nodes_or_with_box(mfp):
    d = default_desc(mfp)
    d.mapping = mfp.MFP_MAP_NODES
    h = ctypes.c_void_p()
    st = mfp.lib().mfp_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == mfp.MFP_ERR_ARG and not h.value
    assert "map_nodes" in mfp.lib().mfp_last_error().decode()
    nodes = (ctypes.c_double * 24)()
    d.map_nodes = ctypes.cast(nodes, ctypes.POINTER(ctypes.c_double))
    d.box_lo = -1.0
    st = mfp.lib().mfp_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == mfp.MFP_ERR_ARG and not h.value
    assert "box" in mfp.lib().mfp_last_error().decode()


def test_neumann_mask(mfp):
    assert mfp.neumann_mask(()) == 0
    assert mfp.neumann_mask((0, 2, 4)) == 0b010101
    assert mfp.neumann_mask([5, 1]) == 0b100010
    with pytest.raises(ValueError):
        mfp.neumann_mask((6,))
