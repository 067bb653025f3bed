"""Accuracy of the GPU path on the benchmark configurations, measured on the device: errors
against closed-form solutions and between the storage precisions (FP64, FP32, BF16-offset).

    python -m paper_2505_17057_gb300.accuracy [--quick] [--case NAME ...]

prints one JSON line per case.  The closed forms are the analytic Taylor-Green decay (the NSE
workloads; velocity error, GRE = sum |u - u*| / sum |u*| over both components) and the exact
solution of the periodic linear CDE for the trigonometric interpolant of the initial field (the
64^2 CDE workload, and the heat equation for the Crank-Nicolson case).  Where no closed form
exists (NCDE, 3D) the FP64 GPU run of the same
configuration is the reference.  The FP64 GPU path itself is checked against the FP64 CPU oracle
by the test suite (1e-12), so its error against a closed form is the scheme's discretisation
error.  --quick runs reduced sizes and step counts.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import configs, inputs, mmfd


def _run(desc_kw, fields, steps, storage, fields_m1=None, flags=0, **extra):
    kw = dict(desc_kw)
    kw["storage"] = storage
    if storage != "fp64" and "ref" not in kw and kw["pde"] != "NSE":
        kw["ref"] = [float(np.mean(fields[0]))]
    s = mmfd.Solver(mmfd.make_desc(**kw, flags=flags, **extra))
    try:
        s.set_fields(fields)
        if fields_m1 is not None:
            s.set_fields(fields_m1, level=1)
        m0 = s.reduce(mmfd.MMFD_RED_SUM)[0]
        s.step(steps)
        out = s.fields(0)
        m1 = s.reduce(mmfd.MMFD_RED_SUM)[0]
    finally:
        s.close()
    # change of sum(phi) (or sum(rho)) relative to sum |phi0|: exact conservation gives rounding only
    return out, (m1 - m0) / max(float(np.abs(fields[0]).sum()), 1e-300)


def _gre(a, b):
    return float(sum(np.abs(x - y).sum() for x, y in zip(a, b)) / sum(np.abs(y).sum() for y in b))


def _maxrel(a, b):
    return float(max(np.abs(x - y).max() for x, y in zip(a, b)) / max(np.abs(y).max() for y in b))


def tgv(n=4096, re=100.0, steps=5000):
    """Taylor-Green vortex (D2Q9 He-Luo NSE, LBGK tau = 1): velocity GRE / max error against the
    analytic decay after `steps` steps, per storage."""
    desc, fields, _ = configs.tgv2d_4096(n=n, re=re, storage="fp64")
    u0 = re * configs.NU_LBGK / n
    _, ue, ve = inputs.taylor_green_2d(n, n, u0, configs.NU_LBGK, float(steps))
    res = {"case": f"tgv2d_{n}", "re": re, "steps": steps, "reference": "analytic Taylor-Green decay"}
    outs = {}
    for st, extra in [("fp64", {}), ("fp32", {}), ("bf16", {}), ("bf16_sr", {"seed": 5})]:
        storage = "bf16" if st.startswith("bf16") else st
        flags = mmfd.MMFD_FLAG_STOCHASTIC_ROUND if st == "bf16_sr" else 0
        out, _ = _run(desc, fields, steps, storage, flags=flags, **extra)
        outs[st] = out
        res[st] = {"gre_u": _gre(out[1:], [ue, ve]), "max_u": _maxrel(out[1:], [ue, ve])}
    for st in ("fp32", "bf16", "bf16_sr"):
        res[st]["gre_ratio_to_fp64"] = res[st]["gre_u"] / res["fp64"]["gre_u"]
        res[st]["max_rel_vs_fp64"] = _maxrel(outs[st][1:], outs["fp64"][1:])
    return res


def cde2d_64():
    """The 64^2 linear CDE (Gaussian hill, 200 steps, FP64) on D2Q5 and D2Q9 against the exact
    solution of the PDE for the periodic interpolant of the initial field."""
    res = {"case": "cde2d_64", "reference": "exact periodic LCDE solution (Fourier)"}
    for lat in ("D2Q5", "D2Q9"):
        desc, fields, steps = configs.cde2d_64(lat)
        flags = mmfd.MMFD_FLAG_DROP_OFFDIAG if lat == "D2Q5" else 0
        out, mass = _run(desc, fields, steps, "fp64", flags=flags)
        phi0 = fields[0]
        K = np.asarray(desc["K"], dtype=float)
        if lat == "D2Q5":
            K = np.diag(np.diag(K))     # the axis lattice carries diag(K) only
        u = desc["u"]
        ky = 2 * np.pi * np.fft.fftfreq(phi0.shape[0])
        kx = 2 * np.pi * np.fft.fftfreq(phi0.shape[1])
        KY, KX = np.meshgrid(ky, kx, indexing="ij")
        expo = 1j * (KX * u[0] + KY * u[1]) + K[0, 0] * KX ** 2 + 2 * K[0, 1] * KX * KY + K[1, 1] * KY ** 2
        exact = np.real(np.fft.ifftn(np.fft.fftn(phi0) * np.exp(-expo * steps * desc["dt"])))
        res[lat] = {"gre": _gre(out, [exact]), "max_rel": _maxrel(out, [exact]), "mass_drift": mass}
    return res


def ncde2d(n=1024, steps=10000):
    """The three-level NCDE workload: FP32 and BF16 (stochastic rounding) against the FP64 GPU run."""
    desc, fields, _ = configs.ncde2d_1024(n=n, storage="fp64")
    ref, m64 = _run(desc, fields, steps, "fp64")
    res = {"case": f"ncde2d_{n}", "steps": steps, "reference": "FP64 GPU run", "fp64": {"mass_drift": m64}}
    for st, flags in [("fp32", 0), ("bf16_sr", mmfd.MMFD_FLAG_STOCHASTIC_ROUND)]:
        out, mass = _run(desc, fields, steps, "bf16" if st == "bf16_sr" else st, flags=flags, seed=7)
        res[st] = {"max_rel_vs_fp64": _maxrel(out, ref), "gre_vs_fp64": _gre(out, ref), "mass_drift": mass}
    return res


def three_d(kind="cde3d", n=512, steps=1000):
    """The 3D workloads: FP32 and BF16-offset against the FP64 GPU run."""
    maker = configs.cde3d_512 if kind == "cde3d" else configs.nse3d_512
    desc, fields, _ = maker(n=n, storage="fp64")
    ref, m64 = _run(desc, fields, steps, "fp64")
    res = {"case": f"{kind}_{n}", "steps": steps, "reference": "FP64 GPU run", "fp64": {"mass_drift": m64}}
    for st in ("fp32", "bf16"):
        out, mass = _run(desc, fields, steps, st)
        res[st] = {"max_rel_vs_fp64": _maxrel(out, ref), "gre_vs_fp64": _gre(out, ref), "mass_drift": mass}
    return res


def _run_fp32_storage_emulated(desc_kw, fields, steps, refs):
    """FP64 arithmetic with FP32 storage: the FP64 solver's levels are rounded to what FP32 storage
    would hold (the offset from refs[f] rounded to FP32, plus refs[f]) -- the initial fields and
    the new level after every step, on the device.  Isolates the storage rounding from the FP32
    arithmetic.  (Setting level 0 of a three-level solver also sets level 1, so level t - dt is
    put back after each step.)"""
    import torch

    def rnd(ts):
        return [((f - r).to(torch.float32).to(torch.float64) + r).contiguous() for f, r in zip(ts, refs)]

    three = desc_kw["levels"] == 3
    s = mmfd.Solver(mmfd.make_desc(**{**desc_kw, "storage": "fp64"}))
    try:
        init = rnd([torch.as_tensor(np.ascontiguousarray(f, dtype=np.float64), device="cuda") for f in fields])
        mmfd.mmfd_set_fields(s.h, 0, [t.data_ptr() for t in init], mmfd.MMFD_DEVICE, mmfd.MMFD_DT_F64)
        for _ in range(steps):
            cur = s.fields(0, device=True) if three else None
            s.step(1)
            new = rnd(s.fields(0, device=True))
            mmfd.mmfd_set_fields(s.h, 0, [t.data_ptr() for t in new], mmfd.MMFD_DEVICE, mmfd.MMFD_DT_F64)
            if three:
                mmfd.mmfd_set_fields(s.h, 1, [t.data_ptr() for t in cur], mmfd.MMFD_DEVICE, mmfd.MMFD_DT_F64)
        return s.fields(0)
    finally:
        s.close()


def attribution(case: str, n: int, steps: int):
    """Where the FP32 error comes from: FP32 storage with FP32 arithmetic (the FP32 solver) and
    FP32 storage with FP64 arithmetic (the FP64 solver rounding its new level to FP32 storage after
    every step), both against the FP64 run, max error relative to the field's max.  For the NCDE
    three-level scheme the level t - dt is the previous (already rounded) level."""
    if case == "ncde2d":
        desc, fields, _ = configs.ncde2d_1024(n=n, storage="fp64")
        refs = [0.0]                      # FP32 NCDE levels hold values
    else:
        desc, fields, _ = configs.tgv2d_4096(n=n, storage="fp64")
        refs = [1.0, 0.0, 0.0]            # FP32 NSE levels hold offsets from rho0
    ref, _ = _run(desc, fields, steps, "fp64")
    full, _ = _run(desc, fields, steps, "fp32")
    stor = _run_fp32_storage_emulated(desc, fields, steps, refs)
    sel = slice(1, None) if case == "tgv2d" else slice(0, None)   # the NSE: velocity, as the accuracy figures
    return {"case": f"{case}_{n}", "steps": steps, "reference": "FP64 GPU run",
            "fields": "velocity" if case == "tgv2d" else "phi",
            "fp32_storage_fp32_arith": _maxrel(full[sel], ref[sel]),
            "fp32_storage_fp64_arith": _maxrel(stor[sel], ref[sel])}


def theta_cn(ns=(64, 128, 256), kx=0.3, ky=0.2, t_end=1.0):
    """Crank-Nicolson (the theta-scheme of Eq. (GCN) with theta = 1/2) on D2Q9 with u = 0 and
    K = diag(kx, ky) on [0, 2 pi)^2, dt proportional to dx (n/4 steps to t_end, up to ~50x the
    explicit scheme's diffusive limit), FP64: max error against the exact heat-equation solution
    sin(x) sin(2y) exp(-(kx + 4 ky) t), and the observed order between successive grids."""
    res = {"case": "theta_cn_d2q9", "reference": "exact heat-equation solution", "runs": []}
    errs = []
    for n in ns:
        dx = 2 * math.pi / n
        steps = n // 4
        dt = t_end / steps
        desc = dict(pde="LCDE", lattice="D2Q9", levels=2, n=[n, n], dt=dt, dx=[dx, dx], K=[[kx, 0.0], [0.0, ky]],
                    u=[0.0, 0.0], targets=[0, -1, -1, 0, 0.5], theta=0.5)
        g = np.arange(n) * dx
        Y, X = np.meshgrid(g, g, indexing="ij")
        phi0 = np.sin(X) * np.sin(2 * Y)
        out, mass = _run(desc, [phi0], steps, "fp64")
        err = float(np.abs(out[0] - phi0 * math.exp(-(kx + 4 * ky) * t_end)).max())
        errs.append(err)
        info = mmfd.mmfd_describe(mmfd.make_desc(**desc, storage="fp64"))
        res["runs"].append({"n": n, "steps": steps, "dt_over_explicit_limit": dt / (dx * dx / (2 * (kx + ky))),
                            "jacobi_sweeps": info.sweeps, "max_err": err, "mass_drift": mass})
    res["orders"] = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    return res


def example3(nxs=(5, 10, 20, 40)):
    """Example 3 of Sec. IV as printed: the wave equation d_t^2 phi = (1/2) lap phi on [0, 1]^2 with
    Dirichlet values of the exact solution exp(x + y + t) set before every step (MMFD_BC_DIRICHLET),
    N_t = 2 N_x, the second level from the printed Taylor start-up; GRE over the interior nodes at
    t = 1 for Cases 1-3 (FP64), next to the values Table 4 prints."""
    cases = {1: ("D2Q5", 3 / 8), 2: ("D2Q9", 3 / 8), 3: ("D2Q9", 1 / 2)}
    printed = {1: [2.86e-4, 6.09e-5, 1.39e-5, 3.30e-6], 2: [6.04e-3, 1.74e-3, 4.55e-4, 1.16e-4],
               3: [3.91e-3, 1.13e-3, 2.97e-4, 7.58e-5]}
    res = {"case": "example3", "reference": "exact solution exp(x + y + t); Table 4 of the paper"}
    for c, (lat, gamma) in cases.items():
        gres = []
        for nx in nxs:
            dx, nt = 1.0 / nx, 2 * nx
            dt = 1.0 / nt
            g = np.arange(nx + 1) * dx
            Y, X = np.meshgrid(g, g, indexing="ij")
            p0 = np.exp(X + Y)
            second = np.zeros_like(p0)
            second[1:-1, :] += p0[2:, :] - 2 * p0[1:-1, :] + p0[:-2, :]
            second[:, 1:-1] += p0[:, 2:] - 2 * p0[:, 1:-1] + p0[:, :-2]
            p1 = p0 + dt * p0 + (dt / (2 * dx)) ** 2 * second
            e1 = np.exp(X + Y + dt)
            for sl in ((0, slice(None)), (-1, slice(None)), (slice(None), 0), (slice(None), -1)):
                p1[sl] = e1[sl]
            s = mmfd.Solver(mmfd.make_desc("LWE", lat, 3, [nx + 1, nx + 1], dt, [dx, dx], K=0.5 * np.eye(2),
                                           storage="fp64", boundary="dirichlet", **mmfd.mmfd_wave_coefficients(gamma)))
            try:
                s.set_fields([p1])
                s.set_fields([p0], level=1)
                for m in range(1, nt):
                    s.set_boundary([np.exp(X + Y + (m + 1) * dt)])
                    s.step(1)
                out = s.fields()[0]
            finally:
                s.close()
            ex = np.exp(X + Y + 1.0)
            gres.append(float(np.abs(out - ex)[1:-1, 1:-1].sum() / np.abs(ex)[1:-1, 1:-1].sum()))
        res[f"case{c}"] = {"nx": list(nxs), "gre": gres, "printed": printed[c][:len(nxs)],
                           "orders": [math.log2(gres[i] / gres[i + 1]) for i in range(len(gres) - 1)]}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--case", nargs="*",
                    default=["cde2d", "tgv100", "tgv1000", "ncde2d", "cde3d", "nse3d", "theta", "example3"])
    args = ap.parse_args()
    q = args.quick
    runs = {
        "cde2d": lambda: cde2d_64(),
        "tgv100": lambda: tgv(512 if q else 4096, 100.0, 1000 if q else 5000),
        "tgv1000": lambda: tgv(512 if q else 4096, 1000.0, 1000 if q else 5000),
        "ncde2d": lambda: ncde2d(256 if q else 1024, 1000 if q else 10000),
        "cde3d": lambda: three_d("cde3d", 128 if q else 512, 200 if q else 1000),
        "nse3d": lambda: three_d("nse3d", 128 if q else 512, 200 if q else 1000),
        "theta": lambda: theta_cn((64, 128) if q else (64, 128, 256)),
        "example3": lambda: example3(),
        "attr_ncde2d": lambda: attribution("ncde2d", 256 if q else 1024, 1000 if q else 10000),
        "attr_tgv2d": lambda: attribution("tgv2d", 512 if q else 4096, 1000 if q else 5000),
    }
    import torch
    torch.cuda.init()
    for c in args.case:
        print(json.dumps(runs[c]()), flush=True)


if __name__ == "__main__":
    main()
