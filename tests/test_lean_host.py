"""Host-side selection of the lean He-Luo NSE form (no GPU): mmfd_describe names the kernel
family mmfd_create would pick.  The lean form needs D2Q9 (any isotropic d_0) or D3Q19 (d_0 = 1/3)
with one speed on every axis: then the uu terms of Eq. (3-3) reduce to |u|^2 and (e_p . u)^2; its streaming
variant needs a momentum set proportional to the scalar one in every level,
(abar-, abar+) = kappa (a+, a-), e.g. LBGK tau = 1 (a = abar = (1, 0, 0))."""
import pytest

from paper_2505_17057_gb300 import mmfd

LBGK = dict(a=(1.0, 0.0, 0.0), abar=(1.0, 0.0, 0.0))
GEN = dict(a=(0.95, 0.1, -0.05), abar=(0.9, 0.2, -0.1))
THREE = dict(a=(7 / 8, 0.0, 1 / 8), ahat=(1 / 8, 0.0, -1 / 8), abar=(0.8, 0.0, 0.2), abarhat=(0.1, 0.0, -0.1))
TRT = dict(a=(1.0, 0.0, -0.2), ahat=(0.0, 0.2, 0.0), abar=(1.0, 0.0, 0.2), abarhat=(0.0, -0.2, 0.0))


def kernel(lat, levels, n, storage="fp32", dx=None, d0=None, pde="NSE", **co):
    dim = 2 if lat == "D2Q9" else 3
    kw = dict(pde=pde, lattice=lat, levels=levels, n=n, dt=1.0, dx=dx or [1.0] * dim, storage=storage, d0=d0, **co)
    if pde == "NSE":
        kw["flags"] = mmfd.MMFD_FLAG_ALLOW_UNSTABLE
    return mmfd.mmfd_describe(mmfd.make_desc(**kw)).kernel.decode()


@pytest.mark.parametrize("lat,n", [("D2Q9", [256, 64]), ("D3Q19", [128, 16, 8])])
def test_lean_variants_selected(lat, n):
    d = len(n)
    assert kernel(lat, 2, n, **LBGK) == f"k_march{d}d_nse_s"
    assert kernel(lat, 2, n, storage="bf16", **LBGK) == f"k_march{d}d_nse_s"
    assert kernel(lat, 2, n, **GEN) == f"k_march{d}d_nse_g"
    assert kernel(lat, 3, n, **THREE) == f"k_march{d}d_nse_g"
    assert kernel(lat, 3, n, **TRT) == f"k_march{d}d_nse_s"


@pytest.mark.parametrize("lat,n", [("D2Q9", [256, 64]), ("D3Q19", [128, 16, 8])])
def test_general_pair_form_where_the_shape_fails(lat, n):
    d = len(n)
    # unequal speeds per axis, d_0 != 1/3, FP64 storage: the general pair form
    assert kernel(lat, 2, n, dx=[1.0, 1.1, 0.9][:d], **LBGK) == f"k_march{d}d"
    # d_0 != 1/3: on D3Q19 the diagonal pairs' cross terms no longer match (e_p . u)^2; D2Q9's
    # diagonal pairs have no third axis and keep the shape for any isotropic d_0
    want = "k_march2d_nse_s" if d == 2 else "k_march3d"
    assert kernel(lat, 2, n, d0=[0.3] * d, **LBGK) == want
    assert kernel(lat, 2, n, storage="fp64", **LBGK) == f"k_march{d}d"
    # narrow grids take the direct kernel whatever the form
    small = [64] + n[1:]
    assert kernel(lat, 2, small, **LBGK) == "k_direct"


def test_other_pdes_use_the_general_kernels():
    assert kernel("D2Q9", 2, [256, 64], pde="LCDE", K=[[0.02, 0], [0, 0.02]], u=[0.1, 0.0],
                  targets=[0, -1, -1, 0, 0.5]) == "k_march2d"
    assert kernel("D3Q19", 2, [128, 8, 8], pde="NCDE", flux=[[0, 0.05, 0.1, 0]] * 3, diff=[0.15, 0, 0.05, 0],
                  a=(0.95, 0.1, -0.05)) == "k_march3d"


def info(lat, levels, n, storage="fp32", pde="NSE", **co):
    dim = len(n)
    kw = dict(pde=pde, lattice=lat, levels=levels, n=n, dt=1.0, dx=[1.0] * dim, storage=storage, **co)
    if pde == "NSE":
        kw["flags"] = mmfd.MMFD_FLAG_ALLOW_UNSTABLE
    return mmfd.mmfd_describe(mmfd.make_desc(**kw))


def test_3d_lean_tile_rows():
    # 16-row tiles at one CTA per SM where the grid has enough of them (x strips x 16-row tiles x
    # 32-plane segments >= 256, ny >= 128), 4-row tiles at four CTAs per SM otherwise
    assert info("D3Q19", 2, [512, 512, 512], **LBGK).tile_rows == 16
    assert info("D3Q19", 2, [512, 512, 512], storage="bf16", **LBGK).tile_rows == 16
    assert info("D3Q19", 3, [384, 384, 384], **THREE).tile_rows == 16
    assert info("D3Q19", 2, [256, 256, 256], **GEN).tile_rows == 16
    assert info("D3Q19", 2, [128, 128, 128], **LBGK).tile_rows == 4
    assert info("D3Q19", 2, [512, 64, 512], **LBGK).tile_rows == 4      # ny < 128
    assert info("D3Q19", 2, [256, 256, 16], **LBGK).tile_rows == 4      # too few planes
    # the general pair form, FP64 storage and the scalar PDEs keep their tiles; 2D reports none
    assert info("D3Q19", 2, [512, 512, 512], storage="fp64", **LBGK).tile_rows == 4
    assert info("D3Q7", 2, [256, 256, 256], pde="LCDE", K=[[0.01, 0, 0], [0, 0.01, 0], [0, 0, 0.01]],
                u=[0.01, 0.0, 0.0], targets=[0, -1, -1, 0, 0.5]).tile_rows == 8
    assert info("D2Q9", 2, [4096, 4096], **LBGK).tile_rows == 0
