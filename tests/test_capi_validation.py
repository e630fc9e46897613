"""Argument checking of the C ABI (host logic, no GPU): every rejected call returns its error code
and message before any CUDA call, so these run on a machine without a GPU.

Covers the degenerate inputs: empty grids, grids whose padded size overflows the 32-bit cell
index, colatitude ranges whose ghost cells reach a pole, boundary codes on the wrong face, bad
physics and numerics options, NULL contexts and negative step counts."""
import ctypes as C
import math

import pytest

from paper_2501_15923_gb300 import inputs as I

EINVAL = -1


@pytest.fixture(scope="module")
def ic():
    from paper_2501_15923_gb300 import build
    build.build()
    from paper_2501_15923_gb300 import icarus
    return icarus


def init_rc(ic, grid, gamma=1.5, opts=None, precision=0):
    lib = ic.load()
    o = ic.make_options(opts or I.Options(), precision)
    ctx = C.c_void_p()
    rc = lib.icarus_init(C.byref(ic.make_grid(grid)), gamma, 0.0, C.byref(o), C.byref(ctx))
    return rc, lib.icarus_last_error().decode(), ctx


def sph(n1=8, n2=12, n3=8, **kw):
    g = I.Grid(n1, n2, n3)
    for k, v in kw.items():
        setattr(g, k, v)
    return g


@pytest.mark.parametrize("grid,msg", [
    (sph(0, 12, 8), "cell counts"),
    (sph(8, 0, 8), "cell counts"),
    (sph(8, 12, 0), "cell counts"),
    (sph(2000, 2000, 1000), "too large"),
    (sph(geometry=7), "geometry"),
    (sph(x1min=2.0, x1max=1.0), "empty coordinate range"),
    (sph(x1min=0.0), "r_in"),
    (sph(x2min=0.05, x2max=math.pi - 0.05), "colatitude"),
    (sph(band_refine=65, band_lo=0.5, band_hi=1.0), "band_refine"),
    (sph(band_refine=-1), "band_refine"),
    (sph(band_refine=4, band_lo=0.05, band_hi=1.0), "band"),
    (sph(band_refine=4, band_lo=1.0, band_hi=0.5), "band"),
    (sph(band_refine=4, band_lo=1.0, band_hi=2.0), "band"),
])
def test_bad_grids_rejected(ic, grid, msg):
    rc, err, ctx = init_rc(ic, grid)
    assert rc == EINVAL and msg in err, (rc, err)
    assert not ctx.value
    # the allocation-free time step accepts exactly the grids icarus_init accepts (rejected before
    # any CUDA call; the pointers are never dereferenced)
    lib = ic.load()
    rc = lib.icarus_cfl_dt_noalloc(C.byref(ic.make_grid(grid)), 1.5, 0.8, C.c_void_p(16), C.c_void_p(16), None)
    assert rc == EINVAL and msg in lib.icarus_last_error().decode()


def test_bad_boundary_codes_rejected(ic):
    g = sph()
    g.bc = (I.BC_DRIVEN, I.BC_DRIVEN, I.BC_CONT, I.BC_CONT, I.BC_PERIODIC, I.BC_PERIODIC)
    rc, err, _ = init_rc(ic, g)
    assert rc == EINVAL and "DRIVEN" in err
    g.bc = (I.BC_DRIVEN, I.BC_CONT, I.BC_CONT, I.BC_CONT, 9, I.BC_PERIODIC)
    rc, err, _ = init_rc(ic, g)
    assert rc == EINVAL and "boundary code" in err
    g = sph(n3=1)
    g.bc = (I.BC_DRIVEN, I.BC_CONT, I.BC_CONT, I.BC_CONT, I.BC_REFLECT, I.BC_REFLECT)
    rc, err, _ = init_rc(ic, g)
    assert rc == EINVAL and "REFLECT" in err


@pytest.mark.parametrize("gamma,opts,precision,msg", [
    (1.0, I.Options(), 0, "gamma"),
    (1.5, I.Options(cfl=0.0), 0, "cfl"),
    (1.5, I.Options(cfl=1.5), 0, "cfl"),
    (1.5, I.Options(limiter=3), 0, "limiter"),
    (1.5, I.Options(flux=3), 0, "flux"),
    (1.5, I.Options(divb=-1), 0, "divb"),
    (1.5, I.Options(init_vphi=2), 0, "init_vphi"),
    (1.5, I.Options(cme_model=2), 0, "cme_model"),
    (1.5, I.Options(tracer=2), 0, "tracer"),
    (1.5, I.Options(strict_floors=2), 0, "strict_floors"),
    (1.5, I.Options(divb=4), 0, "divb"),
    (1.5, I.Options(divb=I.DIVB_GLM, glm_alpha=-1.0), 0, "glm_alpha"),
    (1.5, I.Options(), 3, "precision"),
])
def test_bad_options_rejected(ic, gamma, opts, precision, msg):
    rc, err, _ = init_rc(ic, sph(), gamma, opts, precision)
    assert rc == EINVAL and msg in err, (rc, err)


def test_fused_stage_rejects_hlld(ic):
    lib = ic.load()
    o = ic.make_options(I.Options(flux=I.FLUX_HLLD), 1, fused=True)
    ctx = C.c_void_p()
    rc = lib.icarus_init(C.byref(ic.make_grid(sph())), 1.5, 0.0, C.byref(o), C.byref(ctx))
    assert rc == EINVAL and "fused" in lib.icarus_last_error().decode()


@pytest.mark.parametrize("fused", [-1, 3])
def test_fused_option_out_of_range(ic, fused):
    lib = ic.load()
    o = ic.make_options(I.Options(), 2, fused=fused)
    ctx = C.c_void_p()
    rc = lib.icarus_init(C.byref(ic.make_grid(sph())), 1.5, 0.0, C.byref(o), C.byref(ctx))
    assert rc == EINVAL and "fused" in lib.icarus_last_error().decode()


def test_fused_stage_rejects_glm(ic):
    lib = ic.load()
    o = ic.make_options(I.Options(divb=I.DIVB_GLM), 1, fused=True)
    ctx = C.c_void_p()
    rc = lib.icarus_init(C.byref(ic.make_grid(sph())), 1.5, 0.0, C.byref(o), C.byref(ctx))
    assert rc == EINVAL and "GLM" in lib.icarus_last_error().decode()


def test_fused_stage_and_batch_reject_powell(ic):
    lib = ic.load()
    o = ic.make_options(I.Options(divb=I.DIVB_POWELL), 2, fused=True)
    ctx = C.c_void_p()
    rc = lib.icarus_init(C.byref(ic.make_grid(sph())), 1.5, 0.0, C.byref(o), C.byref(ctx))
    assert rc == EINVAL and "Powell" in lib.icarus_last_error().decode()
    o = ic.make_options(I.Options(divb=I.DIVB_POWELL), 2)
    grids = (ic.icarus_grid * 1)(ic.make_grid(sph()))
    b = C.c_void_p()
    rc = lib.icarus_batch_init(1, C.cast(grids, C.c_void_p), 1.5, 0.0, C.byref(o), C.byref(b))
    assert rc == EINVAL and "Powell" in lib.icarus_last_error().decode()


def test_fused_stage_rejects_tracer(ic):
    lib = ic.load()
    o = ic.make_options(I.Options(tracer=1), 2, fused=True)
    ctx = C.c_void_p()
    rc = lib.icarus_init(C.byref(ic.make_grid(sph())), 1.5, 0.0, C.byref(o), C.byref(ctx))
    assert rc == EINVAL and "tracer" in lib.icarus_last_error().decode()


def test_null_context_and_negative_counts(ic):
    lib = ic.load()
    assert lib.icarus_step(None, 1) == EINVAL
    assert lib.icarus_set_boundary(None, 1, None, None, 0, None) == EINVAL
    assert lib.icarus_sample(None, 1, 1, None, None, 1, None) == EINVAL
    o = ic.make_options(I.Options())
    assert lib.icarus_init(None, 1.5, 0.0, C.byref(o), None) == EINVAL
    assert "NULL" in lib.icarus_last_error().decode()


def test_step_recover_rejects_bad_arguments(ic):
    lib = ic.load()
    h = C.c_int(7)
    assert lib.icarus_step_recover(None, -1, 3, C.byref(h)) == EINVAL and h.value == 0
    assert "n must be" in lib.icarus_last_error().decode()
    for bad in (-1, 21):
        assert lib.icarus_step_recover(None, 1, bad, None) == EINVAL
        assert "max_retries" in lib.icarus_last_error().decode()
    assert lib.icarus_step_recover(None, 1, 3, None) == EINVAL
    assert "NULL context" in lib.icarus_last_error().decode()


def test_barrier_selftest_rejects_bad_arguments(ic):
    """The barrier self-test checks its sizes before any device call."""
    lib = ic.load()
    for blocks, absent, spin in [(0, -1, 1000), (65, -1, 1000), (4, 4, 1000), (4, -1, 0)]:
        assert lib.icarus_batch_barrier_selftest(blocks, absent, spin) == EINVAL


def test_closure_wait_selftest_rejects_bad_arguments(ic):
    lib = ic.load()
    for arrive, limit in [(2, 100), (-1, 100), (1, 0)]:
        assert lib.icarus_closure_wait_selftest(arrive, limit) == EINVAL


def test_math_check_rejects_bad_arguments(ic):
    lib = ic.load()
    x = (C.c_double * 2)(1.0, 4.0)
    y = (C.c_double * 8)()
    assert lib.icarus_math_check(0, x, y) == EINVAL
    assert lib.icarus_math_check(2, None, y) == EINVAL
    assert lib.icarus_math_check(2, x, None) == EINVAL


def test_fma_rate_rejects_bad_arguments(ic):
    """The FMA-rate measurement's argument checks (no GPU needed: rejected before any CUDA call)."""
    lib = ic.load()
    tf, ms = C.c_double(), C.c_double()
    for args in ((3, 8, 4, 16), (0, 3, 4, 16), (0, 8, 0, 16), (0, 8, 9, 16), (1, 8, 4, 6), (1, 8, 4, 0)):
        assert lib.icarus_fma_rate(*args, C.byref(tf), C.byref(ms)) == EINVAL, args
    assert lib.icarus_fma_rate(0, 8, 4, 16, None, C.byref(ms)) == EINVAL
