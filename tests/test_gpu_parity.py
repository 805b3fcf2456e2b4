"""GPU (libsmi, FP32) against the FP64 CPU oracle, through the C ABI.

Bars: computing-box bounds bit-exact; seismograms within 1e-4 relative L2;
RTM images and FWI gradients within 1e-3 relative L2 with FP32 saved
boundaries.  The misfit bar follows from the seismogram bar: with
J = 1/2 |r|^2 and r = u - d, a seismogram error du moves J by at most
|r| |du| + |du|^2 / 2, so |J - J_ref| <= 1e-4 |u_ref| |r_ref| (1 + 1e-4).  16-bit boundary storage reports
its own measured error.  Cases span several thread blocks, ragged box
edges, off-node sources and receivers (Kaiser-sinc stencils), orders 4
and 8, 2D and 3D, with the computing box on and off.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_02293_gb300 import synth as S

pytestmark = pytest.mark.gpu

SEIS_TOL = 1e-4
IMG_TOL = 1e-3


@pytest.fixture(scope="module")
def smi():
    import torch
    from paper_2311_02293_gb300 import build
    build.build()
    from paper_2311_02293_gb300 import smi as mod
    torch.cuda.init()
    return mod


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gprob(smi, w, **kw):
    args = dict(order=w.order, nb=w.nb)
    args.update(kw)
    return smi.Problem(w.d, w.nt, w.dt, w.fm, **args)


def _oprob(w, **kw):
    args = dict(order=w.order, nb=w.nb, fm=w.fm)
    args.update(kw)
    return O.Problem(w.n, w.d, w.nt, w.dt, **args)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


SMALL = {
    "2d_o4_off": lambda: S.tiny_2d(nz=50, nx=44, nt=150, nb=8, src=(9, 21), off_grid=True),
    "2d_o8_on": lambda: S.tiny_2d(nz=45, nx=61, nt=160, nb=10, order=8, src=(12, 30)),
    "3d_o4_off": lambda: S.tiny_3d(nz=30, nx=26, ny=22, nt=70, nb=6, off_grid=True),
    "3d_o8_on": lambda: S.tiny_3d(nz=28, nx=24, ny=26, nt=60, nb=8, order=8),
}


# 3D runs the two-pass tile kernels with the CPML band kernels by default;
# "fused" runs the single-pass step (velocity and pressure in one kernel, CPML
# inline), "inline" the two-pass kernels with the CPML terms in a band-tile
# class.
KERNELS = {"2d_o4_off": ["auto"], "2d_o8_on": ["auto"], "3d_o4_off": ["auto", "fused", "inline"],
           "3d_o8_on": ["auto", "fused", "inline"]}
CASE_KERNELS = [(c, k) for c in sorted(SMALL) for k in KERNELS[c]]


@pytest.mark.parametrize("case,kernels", CASE_KERNELS)
@pytest.mark.parametrize("use_box", [True, False])
def test_forward_parity(smi, case, kernels, use_box):
    w = SMALL[case]()
    seis = smi.smi_forward(_dev(w.vp), _dev(w.rho), _gprob(smi, w, use_box=use_box, kernels=kernels), w.srcs,
                           w.recs, _dev(w.stf))[0].cpu().numpy()
    ref = O.forward(_oprob(w, use_box=use_box), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    assert _rel(seis, ref) <= SEIS_TOL


def test_forward_parity_two_layer_2d_full_size(smi):
    """201 x 201, order 4, nt = 1000, 201 surface receivers (the 2D forward
    workload), all samples compared."""
    w = S.two_layer_2d()
    seis = smi.smi_forward(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs,
                           _dev(w.stf))[0].cpu().numpy()
    ref = O.forward(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    print(f"2D two-layer 201x201 forward: seismograms {_rel(seis, ref):.2e}")
    assert _rel(seis, ref) <= SEIS_TOL


@pytest.mark.parametrize("which", ["source", "receivers"])
@pytest.mark.parametrize("case", ["2d_o4_off", "3d_o8_on"])
def test_box_bounds_bit_exact(smi, case, which):
    w = SMALL[case]()
    prob = _gprob(smi, w)
    n0, count = -1, w.nt + 5
    lo, hi = smi.smi_box_table(_dev(w.vp), _dev(w.rho), prob, w.srcs, w.recs, _dev(w.stf), 0,
                               which, n0, count)
    pts = w.srcs[0] if which == "source" else w.recs[0]
    rlo, rhi = O.box_table(_oprob(w), w.vp, w.rho, pts, n0, count)
    # the oracle marks an empty box by hi < lo on every axis, like the library
    assert np.array_equal(lo, rlo) and np.array_equal(hi, rhi)


def test_box_bounds_bit_exact_3d_corner_source_full_grid(smi):
    """The 400 x 400 x 200 random-medium geometry (corner source, 200 x 200
    receiver carpet): every step of nt = 3000, source and receiver boxes."""
    w = S.random_smooth_3d(nt=3000)
    prob = _gprob(smi, w)
    for which, pts in (("source", w.srcs[0]), ("receivers", w.recs[0])):
        lo, hi = smi.smi_box_table(_dev(w.vp), _dev(w.rho), prob, w.srcs, w.recs, _dev(w.stf), 0,
                                   which, 0, w.nt)
        rlo, rhi = O.box_table(_oprob(w), w.vp, w.rho, pts, 0, w.nt)
        assert np.array_equal(lo, rlo) and np.array_equal(hi, rhi)


def _misfit_ok(J, Jr, seis_ref):
    bound = SEIS_TOL * np.linalg.norm(seis_ref) * np.sqrt(2.0 * Jr) * (1 + SEIS_TOL)
    return abs(J - Jr) <= bound


def _observed(w, scale=0.8):
    """Observed data from the oracle (never from the GPU path): a scaled
    copy of the oracle's seismograms plus seeded noise."""
    ref = O.forward(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    rng = np.random.default_rng(7)
    return (scale * ref + 0.02 * np.abs(ref).max() * rng.standard_normal(ref.shape)).astype(np.float32)


@pytest.mark.parametrize("case,kernels", CASE_KERNELS)
@pytest.mark.parametrize("use_box", [True, False])
def test_gradient_parity(smi, case, kernels, use_box):
    w = SMALL[case]()
    dobs = _observed(w)
    J, g = smi.smi_fwi_gradient(_dev(w.vp), _dev(w.rho), _gprob(smi, w, use_box=use_box, kernels=kernels), w.srcs,
                                w.recs, _dev(w.stf), _dev(dobs))
    Jr, gr, ur = O.gradient(_oprob(w, use_box=use_box), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert _misfit_ok(float(J.item()), Jr, ur)
    assert _rel(g.cpu().numpy(), gr) <= IMG_TOL


@pytest.mark.parametrize("case,kernels", CASE_KERNELS)
def test_rtm_parity(smi, case, kernels):
    w = SMALL[case]()
    dobs = _observed(w, scale=1.0)
    img = smi.smi_rtm(_dev(w.vp), _dev(w.rho), _gprob(smi, w, kernels=kernels), w.srcs, w.recs, _dev(w.stf),
                      _dev(dobs))
    _, ir, _ = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode="rtm")
    assert _rel(img.cpu().numpy(), ir) <= IMG_TOL


@pytest.mark.parametrize("prec,tol", [("f16", 5e-3), ("bf16", 3e-2)])
def test_16bit_boundaries_report_their_error(smi, prec, tol):
    w = SMALL["2d_o8_on"]()
    dobs = _observed(w)
    _, g32 = smi.smi_fwi_gradient(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs,
                                  _dev(w.stf), _dev(dobs))
    _, g16 = smi.smi_fwi_gradient(_dev(w.vp), _dev(w.rho), _gprob(smi, w, shell_prec=prec),
                                  w.srcs, w.recs, _dev(w.stf), _dev(dobs))
    _, gr, _ = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    e16 = _rel(g16.cpu().numpy(), gr)
    e32 = _rel(g32.cpu().numpy(), gr)
    print(f"{prec} boundary storage: gradient error {e16:.2e} (FP32 storage {e32:.2e})")
    assert e16 <= tol


def test_host_pointers_match_device_pointers(smi):
    w = SMALL["2d_o4_off"]()
    prob = _gprob(smi, w)
    d = smi.smi_forward(_dev(w.vp), _dev(w.rho), prob, w.srcs, w.recs, _dev(w.stf))[0].cpu().numpy()
    h = smi.smi_forward(w.vp, w.rho, prob, w.srcs, w.recs, w.stf)[0]
    assert isinstance(h, np.ndarray) and np.array_equal(d, h)
    dobs = _observed(w)
    Jd, gd = smi.smi_fwi_gradient(_dev(w.vp), _dev(w.rho), prob, w.srcs, w.recs, _dev(w.stf), _dev(dobs))
    Jh, gh = smi.smi_fwi_gradient(w.vp, w.rho, prob, w.srcs, w.recs, w.stf, dobs)
    assert float(Jd.item()) == float(Jh[0]) and np.array_equal(gd.cpu().numpy(), gh)


def test_shot_batching_is_bitwise_invariant(smi):
    """Shots propagated together or one at a time give identical results."""
    base = S.layered_fault_2d(nz=60, nx=140, nt=300, nshot=4, order=4)
    base.srcs[:, 1] = [200.0, 600.0, 1000.0, 1500.0]
    prob_all = _gprob(smi, base)
    prob_one = _gprob(smi, base, max_batch=1)
    vp, rho, stf = _dev(base.vp), _dev(base.rho), _dev(base.stf)
    a = smi.smi_forward(vp, rho, prob_all, base.srcs, base.recs, stf, flat=True)
    b = smi.smi_forward(vp, rho, prob_one, base.srcs, base.recs, stf, flat=True)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    dobs = 0.5 * a
    ga = smi.smi_fwi_gradient(vp, rho, prob_all, base.srcs, base.recs, stf, dobs)[1]
    gb = smi.smi_fwi_gradient(vp, rho, prob_one, base.srcs, base.recs, stf, dobs)[1]
    assert np.array_equal(ga.cpu().numpy(), gb.cpu().numpy())


def test_multi_shot_gradient_sums_single_shots(smi):
    base = S.layered_fault_2d(nz=50, nx=120, nt=250, nshot=3, order=4)
    base.srcs[:, 1] = [150.0, 700.0, 1300.0]
    prob = _gprob(smi, base)
    vp, rho, stf = _dev(base.vp), _dev(base.rho), _dev(base.stf)
    seis = smi.smi_forward(_dev(base.vp_true), rho, prob, base.srcs, base.recs, stf)
    J, g = smi.smi_fwi_gradient(vp, rho, prob, base.srcs, base.recs, stf, seis)
    Js, gs = 0.0, 0.0
    for s in range(3):
        j, gg = smi.smi_fwi_gradient(vp, rho, prob, base.srcs[s:s + 1], base.recs[s:s + 1], stf, seis[s])
        Js += float(j.item())
        gs = gs + gg.cpu().numpy().astype(np.float64)
    assert abs(float(J.item()) - Js) <= 1e-12 * Js
    assert _rel(g.cpu().numpy(), gs) <= 1e-6


def test_gradient_parity_layered_fault_2d_full_grid(smi):
    """Full 301 x 1001 grid, order 8, 1001 receivers, one shot of the 40,
    observed data from the oracle on the true model; nt shortened to 500
    so that the FP64 oracle finishes in a test."""
    w = S.layered_fault_2d(nt=500).subset([5])
    dobs = O.forward(_oprob(w), w.vp_true, w.rho, w.stf, w.srcs[0], w.recs[0]).astype(np.float32)
    J, g = smi.smi_fwi_gradient(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs,
                                _dev(w.stf), _dev(dobs))
    Jr, gr, ur = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    print(f"2D layered-fault 301x1001 gradient: {_rel(g.cpu().numpy(), gr):.2e}, "
          f"misfit {abs(float(J.item()) - Jr) / Jr:.2e}")
    assert _misfit_ok(float(J.item()), Jr, ur)
    assert _rel(g.cpu().numpy(), gr) <= IMG_TOL


def test_errors_are_reported(smi):
    w = SMALL["2d_o4_off"]()
    with pytest.raises(smi.SmiError) as e:
        smi.smi_forward(_dev(w.vp), _dev(w.rho), smi.Problem(w.d, w.nt, 5e-3, w.fm, nb=8), w.srcs,
                        w.recs, _dev(w.stf))
    assert e.value.code == -2
    with pytest.raises(smi.SmiError) as e:
        smi.smi_forward(_dev(w.vp), _dev(w.rho), smi.Problem(w.d, w.nt, w.dt, 60.0, nb=8), w.srcs,
                        w.recs, _dev(w.stf))
    assert e.value.code == -3
    bad = w.srcs.copy()
    bad[0, 0] = -100.0
    with pytest.raises(smi.SmiError) as e:
        smi.smi_forward(_dev(w.vp), _dev(w.rho), _gprob(smi, w), bad, w.recs, _dev(w.stf))
    assert e.value.code == -1
    vp = w.vp.copy()
    vp[3, 3] = -1.0
    with pytest.raises(smi.SmiError) as e:
        smi.smi_forward(_dev(vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf))
    assert e.value.code == -1


@pytest.mark.parametrize("order,kernels", [(4, "auto"), (8, "auto"), (4, "fused"), (8, "fused"), (4, "inline"),
                                           (8, "inline")])
def test_long_adjoint_through_cpml_corners_3d(smi, order, kernels):
    """Hundreds of steps with most of the energy inside the CPML slabs and
    their edges/corners: the transposed CPML terms of the adjoint must stay
    exact there (an inexact transpose drifts and can become unstable)."""
    w = S.tiny_3d(nz=18, nx=16, ny=14, nt=450, nb=8, order=order, off_grid=True)
    dobs = _observed(w)
    J, g = smi.smi_fwi_gradient(_dev(w.vp), _dev(w.rho), _gprob(smi, w, kernels=kernels), w.srcs, w.recs,
                                _dev(w.stf), _dev(dobs))
    Jr, gr, ur = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert _misfit_ok(float(J.item()), Jr, ur)
    assert _rel(g.cpu().numpy(), gr) <= IMG_TOL
    img = smi.smi_rtm(_dev(w.vp), _dev(w.rho), _gprob(smi, w, kernels=kernels), w.srcs, w.recs, _dev(w.stf),
                      _dev(dobs))
    _, ir, _ = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode="rtm")
    assert _rel(img.cpu().numpy(), ir) <= IMG_TOL


@pytest.mark.parametrize("case", ["2d_o8_on", "3d_o8_on"])
def test_normalised_rtm_image_parity(smi, case):
    """Normalised imaging condition (Sec. 2.3): per-shot image over the
    shot's source illumination, summed over shots; two shots so that the
    normalisation is per shot."""
    w = SMALL[case]()
    moved = w.srcs.copy()
    moved[:, 1] += 3 * w.d[1]                          # a second shot 3 cells along x
    srcs = np.concatenate([w.srcs, moved])
    recs = [w.recs[0], w.recs[0]]
    dobs = [O.forward(_oprob(w), w.vp, w.rho, w.stf, s, recs[0]) for s in srcs]
    img = smi.smi_rtm(_dev(w.vp), _dev(w.rho), _gprob(smi, w, img_norm=True), srcs, recs, _dev(w.stf),
                      [_dev(d.astype(np.float32)) for d in dobs])
    ref = sum(O.gradient(_oprob(w), w.vp, w.rho, w.stf, s, recs[0], d, mode="rtm_norm")[1] for s, d in zip(srcs, dobs))
    assert _rel(img.cpu().numpy(), ref) <= IMG_TOL


@pytest.mark.parametrize("case", sorted(SMALL))
def test_generic_kernels_parity(smi, case):
    """The generic grid-stride kernels (opts.kernels = SMI_KERNELS_GENERIC:
    the path of 3D fields of 2^31 points or more and of
    smi_forward_noalloc, CPML inline) against the oracle: seismograms, FWI
    gradient, misfit and RTM image."""
    w = SMALL[case]()
    vp, rho, stf = _dev(w.vp), _dev(w.rho), _dev(w.stf)
    prob = _gprob(smi, w, kernels="generic")
    seis = smi.smi_forward(vp, rho, prob, w.srcs, w.recs, stf)[0].cpu().numpy()
    ref = O.forward(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    assert _rel(seis, ref) <= SEIS_TOL
    dobs = _observed(w)
    J, g = smi.smi_fwi_gradient(vp, rho, prob, w.srcs, w.recs, stf, _dev(dobs))
    Jr, gr, ur = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert _misfit_ok(float(J.item()), Jr, ur)
    assert _rel(g.cpu().numpy(), gr) <= IMG_TOL
    img = smi.smi_rtm(vp, rho, prob, w.srcs, w.recs, stf, _dev(dobs))
    _, ir, _ = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode="rtm")
    assert _rel(img.cpu().numpy(), ir) <= IMG_TOL


@pytest.mark.parametrize("order", [4, 8])
def test_generic_kernels_box_off_long_3d(smi, order):
    """The generic adjoint and reconstruction kernels with the box off over
    hundreds of steps, energy in the CPML slabs and corners."""
    w = S.tiny_3d(nz=18, nx=16, ny=14, nt=300, nb=8, order=order, off_grid=True)
    dobs = _observed(w)
    prob = _gprob(smi, w, kernels="generic", use_box=False)
    J, g = smi.smi_fwi_gradient(_dev(w.vp), _dev(w.rho), prob, w.srcs, w.recs, _dev(w.stf), _dev(dobs))
    Jr, gr, ur = O.gradient(_oprob(w, use_box=False), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert _misfit_ok(float(J.item()), Jr, ur)
    assert _rel(g.cpu().numpy(), gr) <= IMG_TOL


def test_16bit_boundaries_3d_against_the_oracle(smi):
    """FP16 / BF16 boundary storage in 3D (salt model at 60^3 + 20 CPML
    layers, order 8, 200 steps, one shot): the image and gradient error of
    each storage precision measured against the FP64 oracle itself (not
    against FP32 storage).  Bars as in 2D; the measured values are printed."""
    w = S.salt_3d(n=60, nt=200, nshot=1)
    w.stf = S.ricker(w.nt + 40, w.dt, w.fm)[40:].copy()
    dobs = _observed(w)
    vp, rho, stf, d = _dev(w.vp), _dev(w.rho), _dev(w.stf), _dev(dobs)
    _, gr, _ = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    _, ir, _ = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode="rtm")
    for prec, tol in (("f32", IMG_TOL), ("f16", 5e-3), ("bf16", 3e-2)):
        prob = _gprob(smi, w, shell_prec=prec)
        _, g = smi.smi_fwi_gradient(vp, rho, prob, w.srcs, w.recs, stf, d)
        img = smi.smi_rtm(vp, rho, prob, w.srcs, w.recs, stf, d)
        eg, ei = _rel(g.cpu().numpy(), gr), _rel(img.cpu().numpy(), ir)
        print(f"3D {prec} boundary storage vs oracle: gradient {eg:.2e}, image {ei:.2e}")
        assert eg <= tol and ei <= tol


@pytest.mark.parametrize("order", [4, 8])
@pytest.mark.parametrize("use_box", [True, False])
@pytest.mark.parametrize("other", ["fused", "inline"])
def test_single_pass_matches_two_pass(smi, order, use_box, other):
    """The single-pass 3D step and the inline-CPML two-pass kernels against
    the default two-pass kernels on a grid of several tiles in every
    direction (tile columns in and out of the CPML bands, several y-chunks,
    two shots in one batch): seismograms, gradient and image agree to FP32
    rounding."""
    import torch
    w = S.tiny_3d(nz=70, nx=50, ny=44, nt=160, nb=10, order=order, off_grid=True)
    moved = w.srcs.copy()
    moved[:, 1] += 7 * w.d[1]
    srcs = np.concatenate([w.srcs, moved])
    recs = [w.recs[0], w.recs[0][::2].copy()]
    vp, rho, stf = _dev(w.vp), _dev(w.rho), _dev(w.stf)
    out = {}
    for k in (other, "twopass"):
        prob = _gprob(smi, w, use_box=use_box, kernels=k)
        seis = smi.smi_forward(vp, rho, prob, srcs, recs, stf, flat=True)
        dobs = (0.8 * seis).contiguous()
        dobs[: dobs.numel() // 3] *= 0.5
        J, g = smi.smi_fwi_gradient(vp, rho, prob, srcs, recs, stf, dobs)
        img = smi.smi_rtm(vp, rho, prob, srcs, recs, stf, dobs)
        out[k] = [t.double().cpu().numpy() for t in (seis, g, img)] + [float(J.item())]
        torch.cuda.synchronize()
    for a, b in zip(out[other][:3], out["twopass"][:3]):
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
    assert abs(out[other][3] - out["twopass"][3]) <= 1e-5 * abs(out["twopass"][3])
