"""C-ABI library: loads without a GPU, exports every declared symbol, and its
host-side integer geometry is bit-exact with the oracle. Also the product's host
setup (screens, modal basis) against the oracle."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_1607_07624_gb300 import build
    build.build()
    from paper_1607_07624_gb300 import pas
    return pas


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pas.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pas_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    import ctypes
    names = declared_functions()
    assert len(names) >= 30
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    # the binding covers the whole header with the same names
    assert sorted(lib.EXPORTED) == names


def test_loop_kernel_count_matches_header(lib):
    src = open(os.path.join(ROOT, "include", "pas.h")).read()
    n = int(re.search(r"#define PAS_LOOP_KERNELS (\d+)", src).group(1))
    assert lib.PAS_LOOP_KERNELS == n
    names = [lib.pas_loop_kernel_name(k) for k in range(n)]
    assert all(names) and lib.pas_loop_kernel_name(n) is None


def test_version_and_supported_sizes(lib):
    assert lib.pas_version() >= 100
    for N in (16, 24, 32, 48, 64, 128, 480, 960):
        assert lib.pas_pyr_supported(N)
    assert not lib.pas_pyr_supported(7) and not lib.pas_pyr_supported(1000)


@pytest.mark.parametrize("Np,obs,n_sub", [(64, 0.1, 16), (240, 0.1, 30), (480, 0.1, 96),
                                          (16, 0.1, 4), (24, 0.0, 4), (60, 0.25, 10)])
def test_geometry_bit_exact_with_oracle(lib, Np, obs, n_sub):
    from oracle import optics as op
    m = op.pupil_mask(Np, obs)
    assert np.array_equal(lib.pas_pupil_mask(Np, obs).astype(bool), m)
    assert np.array_equal(lib.pas_pupil_pixels(Np, obs), np.flatnonzero(m.ravel()).astype(np.int32))
    assert np.array_equal(lib.pas_valid_subaps(Np, obs, n_sub), op.valid_subapertures(Np, obs, n_sub))


def test_geometry_rejects_bad_arguments(lib):
    with pytest.raises(lib.PasError) as e:
        lib.pas_valid_subaps(30, 0.1, 0)
    assert e.value.status == lib.PAS_EINVAL
    with pytest.raises(lib.PasError):
        lib.pas_valid_subaps(30, 0.1, 31)
    with pytest.raises(lib.PasError):
        lib.pas_pupil_mask(16, 1.5)


@pytest.mark.parametrize("Np,n_sub", [(30, 7), (128, 20), (320, 60), (50, 7), (64, 16)])
def test_valid_subaps_non_integer_binning_bit_exact(lib, Np, n_sub):
    """Sub-apertures of Np / n_sub pixels, not necessarily an integer: the library's
    integer overlap rule equals the oracle's."""
    from oracle import optics as op
    assert np.array_equal(lib.pas_valid_subaps(Np, 0.1, n_sub), op.valid_subapertures(Np, 0.1, n_sub))


def test_product_screens_match_oracle():
    from oracle import atmosphere as at
    from paper_1607_07624_gb300 import calib
    from synth import get_config
    from synth.configs import with_
    from synth.inputs import screen_white_noise
    cfg = with_(get_config("scao_lbt_240px"), S=256)
    w = [screen_white_noise(256, 3 + l) for l in range(3)]
    a = calib.layer_screens(cfg, w).astype(np.float64)
    b = at.layer_screens_nm(cfg, w)
    assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))


def test_product_basis_matches_oracle():
    from oracle import modal as md
    from oracle import optics as op
    from paper_1607_07624_gb300 import calib
    idx = np.flatnonzero(op.pupil_mask(64, 0.1).ravel())
    assert np.max(np.abs(calib.zernike_basis(64, idx, 100) - md.modal_basis(64, 0.1, 100))) < 1e-9
    for j in range(1, 300):
        assert calib.noll_nm(j) == md.noll_to_nm(j)


def test_zernike_recurrence_matches_the_oracle_polynomials():
    """calib.zernike_raw (Jacobi three-term recurrence, all pixels per azimuthal
    order) against the oracle's Zernike polynomials (its own radial sum) up to
    radial order 20, and high orders against scipy's Jacobi polynomials."""
    import math
    from oracle import modal as md
    from oracle import optics as op
    from paper_1607_07624_gb300 import calib
    from scipy.special import eval_jacobi
    Np = 64
    idx = np.flatnonzero(op.pupil_mask(Np, 0.1).ravel())
    Z = calib.zernike_raw(Np, idx, 230)            # radial orders up to 20
    rho, th = md.pupil_polar(Np)
    rho, th = rho.ravel()[idx], th.ravel()[idx]
    for c, j in enumerate(range(2, 232)):
        # (the oracle's alternating factorial sum loses ~1e-9 by radial order 18)
        assert np.max(np.abs(Z[:, c] - md.zernike(j, rho, th))) < 1e-8, j
    # radial order 88 (the 4000-mode basis): against P_k^(m,0) from scipy
    Zh = calib.zernike_raw(Np, idx, 4000)
    for j in (3990, 3995, 4001):
        n, m = calib.noll_nm(j)
        k = (n - abs(m)) // 2
        r = (-1) ** k * rho ** abs(m) * eval_jacobi(k, abs(m), 0, 1 - 2 * rho * rho)
        ang = 1.0 if m == 0 else (math.sqrt(2) * (np.cos(m * th) if m > 0 else np.sin(-m * th)))
        assert np.max(np.abs(Zh[:, j - 2] - math.sqrt(n + 1) * r * ang)) < 1e-8 * math.sqrt(n + 1), j


def test_product_kl_basis_matches_oracle():
    """calib.kl_basis (half-spectrum real products, MGS Zernikes) against the oracle's
    (full complex spectrum, QR Zernikes): equal variances, and equal modes up to the
    rotation inside groups of equal variance (cos/sin pairs)."""
    from oracle import modal as md
    from oracle import optics as op
    from paper_1607_07624_gb300 import calib
    Np, nm, dx, r0, L0 = 32, 20, 8.0 / 32, 0.15, 25.0
    mask = op.pupil_mask(Np, 0.1)
    pix = np.flatnonzero(mask.ravel())
    K = calib.kl_basis(Np, pix, nm, dx, r0, L0, pad=4)
    M = md.modal_basis(Np, 0.1, nm)
    Ko, w = md.kl_basis(M, md.modal_covariance(M, mask, dx, r0, L0, 4))
    n = pix.size
    Cp = calib.modal_covariance(K, pix, Np, dx, r0, L0, pad=4)
    assert np.max(np.abs(np.diag(Cp) - w)) <= 1e-8 * w[0]
    i = 0
    while i < nm:                                   # groups of (nearly) equal variance
        j = i + 1
        while j < nm and abs(w[j] - w[i]) <= 1e-6 * w[i]:
            j += 1
        Pp = K[:, i:j] @ K[:, i:j].T / n
        Po = Ko[:, i:j] @ Ko[:, i:j].T / n
        assert np.max(np.abs(Pp - Po)) < 1e-7, (i, j)
        if j - i == 1:
            assert np.max(np.abs(K[:, i] - Ko[:, i])) < 1e-6
        i = j


def test_product_source_geometry_matches_oracle():
    """calib's footprint offsets and cone scales against the oracle's; a source below
    a layer is rejected."""
    from oracle import atmosphere as at
    from paper_1607_07624_gb300 import calib
    heights = [0.0, 837.0, 3045.0, 12780.0]
    for rho, phi, dx in ((10.0, 45.0, 0.035), (30.0, -120.0, 8.4 / 240), (0.0, 0.0, 0.1)):
        a = np.array(calib.footprint_offsets_px(heights, rho, phi, dx))
        b = np.array(at.footprint_offsets_px(heights, rho, phi, dx))
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))
    assert calib.footprint_scales(heights, 90000.0) == at.footprint_scales(heights, 90000.0)
    with pytest.raises(ValueError):
        calib.footprint_scales(heights, 12000.0)


@pytest.mark.parametrize("d,n", [(3.0, 5), (2.0, 3), (1.0, 1), (4.0, 8)])
def test_disc_source_points(d, n):
    """calib.disc_source: the grid points of spacing d/n inside the disc of diameter d,
    counted by brute force, symmetric about the centre, equal spacing."""
    from paper_1607_07624_gb300 import calib
    ex, ey = calib.disc_source(d, n)
    h = d / n
    want = sum(1 for i in range(n) for j in range(n)
               if ((i - (n - 1) / 2) * h) ** 2 + ((j - (n - 1) / 2) * h) ** 2 <= (d / 2) ** 2 + 1e-12)
    assert ex.size == ey.size == want
    assert np.all(ex ** 2 + ey ** 2 <= (d / 2) ** 2 + 1e-9)
    assert abs(ex.sum()) < 1e-9 and abs(ey.sum()) < 1e-9
    if n > 1:
        u = np.unique(np.round(ex / h, 9))
        assert np.allclose(np.diff(u), 1.0)


def test_binding_rejects_mismatched_source_arrays(lib):
    """The binding checks the source arrays' lengths before calling the library."""
    with pytest.raises(ValueError):
        lib.pas_pyr_create_extended(None, 16, 32, 4, 2, 1.0, 750.0, 0.0, [0.0, 1.0], [0.0])
    with pytest.raises(ValueError):
        lib.pas_pyr_create_extended(None, 16, 32, 4, 2, 1.0, 750.0, 0.0, [0.0, 1.0], [0.0, 1.0], [1.0])


def test_static_measure_binding_rejects_wrong_tensors_before_the_call():
    """The C call sees raw pointers only: the binding checks dtype, device and size."""
    torch = pytest.importorskip("torch")
    from paper_1607_07624_gb300 import pas
    Np, N, K, n_sub = 32, 64, 8, 8
    opd = torch.zeros(Np, Np)            # host tensor: refused
    fr = torch.zeros(2 * n_sub, 2 * n_sub)
    with pytest.raises(pas.PasError) as e:
        pas.pas_pyr_measure_static(Np, N, K, n_sub, 2.0, 750.0, 0.1, opd, fr)
    assert e.value.status == pas.PAS_EINVAL and "d_opd" in str(e.value)


def test_profile_cases_command_line():
    """The profiling driver's command line parses on a host without a GPU."""
    from paper_1607_07624_gb300 import profile_cases
    with pytest.raises(SystemExit) as e:
        profile_cases.main(["--help"])
    assert e.value.code == 0
