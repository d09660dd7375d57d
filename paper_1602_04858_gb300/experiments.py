"""Robustness of the V-cycle-preconditioned GMRES on binary permeability fields
(synthetic analogues of the experiments of Sec. 4.1, Tables 1 and 2).

The paper's fields exist only as figures, so three seeded binary structures
of the same kinds stand in for them, generated on 128 x 128 cells and refined
(each cell split in 2 x 2 or 4 x 4) to the finer meshes, as the paper does
with its 128 x 128 data:
  foam       -- mostly disconnected irregular islands (``inputs.foam_mask``)
  inclusions -- isolated rectangles (``inputs.inclusions_mask``)
  connected  -- long connected fibre-like inclusions, 20 random walks two
                cells wide (``inputs.channel_mask``)
case (a): the structure has permeability 1 (c = 1) and the rest 1/contrast
(c = contrast); case (b): the roles reversed.

Flow driven by the boundary velocity g = (1, 0), f = 0, Darcy (mu = 0) or
Brinkman (mu = 0.01), RT_0, variable V-cycle with m(J) = 2, GMRES stopped at
a 1e-6 reduction of the residual (Sec. 4.1).  The constant field u_g = g
satisfies the boundary condition, is divergence free, has no jumps and no
gradient, and its Nitsche terms equal those of the data g (eq. (BCh)); so
u = u_g + u_0 where u_0 solves the same problem with homogeneous boundary
values and body force -c g (cellwise constant).  The solves below compute u_0.

    python -m paper_1602_04858_gb300.experiments [--sizes 128,256,512] [--precision fp32]
    python -m paper_1602_04858_gb300.experiments --table4
    python -m paper_1602_04858_gb300.experiments --variants
    python -m paper_1602_04858_gb300.experiments --scale
    python -m paper_1602_04858_gb300.experiments --degrees

Prints one JSON line per solve and a table of GMRES iterations.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, mgdarcy

GEOMETRIES = ("foam", "inclusions", "connected")


def structure(geometry: str, n0: int = 128, seed: int = 11) -> np.ndarray:
    """Binary structure on n0 x n0 cells (bool, axis order (y, x))."""
    if geometry == "foam":
        return inputs.foam_mask(n0, seed)
    if geometry == "inclusions":
        return inputs.inclusions_mask(n0, seed)
    if geometry == "connected":
        return inputs.channel_mask(n0, 20, seed)
    raise KeyError(geometry)


def coefficient(geometry: str, case: str, contrast: float, n: int, n0: int = 128) -> np.ndarray:
    """Zero-order coefficient c per cell of the n x n mesh (n a multiple of n0)."""
    m = inputs.refine_cells(structure(geometry, n0).astype(np.int8), n // n0).astype(bool)
    inside, outside = (1.0, contrast) if case == "a" else (contrast, 1.0)
    return np.where(m, inside, outside).astype(np.float64)


def driven_solve(torch, c: np.ndarray, mu: float, degree: int = 0, g=(1.0, 0.0), tol: float = 1e-6,
                 maxit: int = 400, precision: str = "fp32", n_coarse: int = 4, coarse_avg: int = 0):
    """u_0 of the driven problem (boundary velocity g, f = 0) on the 2-D or 3-D
    mesh of c: GMRES statistics, the solution vector (x of u_0, pressure with
    zero mean) and the handle."""
    d, n = c.ndim, c.shape[0]
    levels = int(np.log2(n // n_coarse)) + 1
    cd = torch.as_tensor(c, device="cuda")
    G = mgdarcy.Multigrid(d, n_coarse, levels, degree, mu, cd, precision=precision, coarse_avg=coarse_avg)
    nu, npr = G.sizes()
    f = torch.stack([-float(g[e]) * cd.reshape(-1) for e in range(d)]).contiguous()
    b = torch.zeros(nu + npr, dtype=torch.float64, device="cuda")
    G.load_vector(f, None, b)
    x = torch.zeros_like(b)
    st, status = G.solve(b[:nu].contiguous(), b[nu:].contiguous(), x, tol=tol, maxit=maxit, check=False)
    return st, x, G


def add_lift(x: np.ndarray, n: int, degree: int = 0, g=(1.0, 0.0)) -> np.ndarray:
    """u = u_g + u_0: every velocity node of component i gets g_i added."""
    d = len(g)
    N = n * (degree + 1)
    nu1 = (N + 1) * N ** (d - 1)
    y = x.copy()
    for e in range(d):
        y[e * nu1:(e + 1) * nu1] += g[e]
    return y


def table4(torch, sizes=(64, 128), precision="fp32", sigma=2.0, seed=7):
    """Analogue of Table 4: 3-D Brinkman (mu = 0.01), RT_0, lognormal c =
    exp(G) with G ~ GRF(sigma, 4 cells) on 64^3 cells refined to the finer
    meshes (contrast max c / min c = 1.3e6 for sigma = 2, seed 7; SPE10 itself
    is not available), boundary data BC1 g = (1, 0, 0) and BC2 g = (0, 1, 0),
    GMRES to 1e-6, 1e-8, 1e-10."""
    base = inputs.lognormal_c(64, 3, sigma, 4.0, seed)
    rows = []
    for n in sizes:
        r = n // 64
        c = np.ascontiguousarray(np.repeat(np.repeat(np.repeat(base, r, 0), r, 1), r, 2))
        for name, g in (("BC1", (1.0, 0.0, 0.0)), ("BC2", (0.0, 1.0, 0.0))):
            for tol in (1e-6, 1e-8, 1e-10):
                st, _, G = driven_solve(torch, c, 0.01, g=g, tol=tol, precision=precision, n_coarse=2)
                rows.append(dict(table=4, n=n, bc=name, tol=tol, iterations=st.iterations,
                                 converged=bool(st.converged), rel_residual=st.rel_residual,
                                 solve_ms=st.solve_ms, contrast=float(c.max() / c.min())))
                print(json.dumps(rows[-1]), flush=True)
                del G
                torch.cuda.empty_cache()
    print("\nTable 4 analogue: GMRES iterations (3-D Brinkman, lognormal c)")
    print("| h | BC1 1e-6 | BC2 1e-6 | BC1 1e-8 | BC2 1e-8 | BC1 1e-10 | BC2 1e-10 |")
    for n in sizes:
        it = {(r_["bc"], r_["tol"]): r_["iterations"] for r_ in rows if r_["n"] == n}
        print(f"| 1/{n} | " + " | ".join(str(it[(b, t)]) for t in (1e-6, 1e-8, 1e-10) for b in ("BC1", "BC2")) + " |")
    return rows


def variants(torch, precision="fp32"):
    """Smoother and cycle variants on two workloads: the paper's symmetric
    multiplicative Schwarz smoother (interior-vertex patches, and with the
    patches of the boundary vertices as well, Sec. 3.3) against additive Schwarz (omega = 1/4,
    every patch on the same residual: one launch per colour and one update per
    step instead of 2C - 1 dependent passes), each in the variable cycle
    (m(J) = 2) and the standard V(2,2) cycle.  Reports GMRES iterations, the
    V-cycle time and the solve time (CUDA events, GB300)."""
    cases = []
    w = inputs.workload("channels_256")
    cases.append(("channels 256^2 RT_1, random load, 1e-8", w["c"], w["mu"], w["degree"], 1e-8, "random"))
    cases.append(("inclusions 512^2 RT_0 Darcy, driven (a) 1e6, 1e-6",
                  coefficient("inclusions", "a", 1e6, 512), 0.0, 0, 1e-6, "driven"))
    rows = []
    for name, c, mu, k, tol, kind in cases:
        n = c.shape[0]
        for smoother, omega, bnd in (("multiplicative", 0.0, False), ("multiplicative, all vertices", 0.0, True),
                                     ("additive", 0.25, False)):
            for cycle, variable in (("variable", True), ("V(2,2)", False)):
                levels = int(np.log2(n // 4)) + 1
                cd = torch.as_tensor(c, device="cuda")
                G = mgdarcy.Multigrid(2, 4, levels, k, mu, cd, precision=precision, variable_cycle=variable,
                                      additive=omega, boundary_patches=bnd)
                nu, npr = G.sizes()
                b = torch.zeros(nu + npr, dtype=torch.float64, device="cuda")
                if kind == "driven":
                    f = torch.stack([-cd.reshape(-1), 0.0 * cd.reshape(-1)]).contiguous()
                    G.load_vector(f, None, b)
                else:
                    b[:nu] = torch.as_tensor(np.random.default_rng(11).standard_normal(nu), device="cuda")
                r = torch.as_tensor(np.random.default_rng(1).standard_normal(nu + npr), device="cuda")
                z = torch.zeros_like(r)
                for _ in range(3):
                    G.vcycle(r, z)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(10):
                    G.vcycle(r, z)
                e1.record()
                torch.cuda.synchronize()
                x = torch.zeros_like(b)
                st, _ = G.solve(b[:nu].contiguous(), b[nu:].contiguous(), x, tol=tol, maxit=400, check=False)
                rows.append(dict(case=name, smoother=smoother, cycle=cycle, iterations=st.iterations,
                                 converged=bool(st.converged), vcycle_ms=e0.elapsed_time(e1) / 10,
                                 solve_ms=st.solve_ms))
                print(json.dumps(rows[-1]), flush=True)
                del G
                torch.cuda.empty_cache()
    print("\n| workload | smoother | cycle | iterations | V-cycle ms | solve ms |")
    for r_ in rows:
        print(f"| {r_['case']} | {r_['smoother']} | {r_['cycle']} | {r_['iterations']}"
              f"{'' if r_['converged'] else ' (not converged)'} | {r_['vcycle_ms']:.2f} | {r_['solve_ms']:.1f} |")
    return rows


def degrees(torch, precision="fp32", sizes=(128, 256)):
    """Polynomial degree (Sec. 2.3 defines RT_k x Q_k for every k): RT_0, RT_1
    and RT_2 on the same meshes and coefficient (20 channels two cells wide,
    contrast 1e6, mu = 0.01, the recipe of the 256^2 benchmark), random load
    in the velocity rows, FGMRES to 1e-8, variable V-cycle with m(J) = 2.
    Reports iterations, V-cycle and solve times (CUDA events) and the V-cycle
    rate in dofs x V-cycles per second."""
    rows = []
    for n in sizes:
        c = inputs.channel_c(n, 20, 2)
        levels = int(np.log2(n // 4)) + 1
        for k in (0, 1, 2):
            cd = torch.as_tensor(c, device="cuda")
            t0 = time.perf_counter()
            G = mgdarcy.Multigrid(2, 4, levels, k, 0.01, cd, precision=precision)
            setup_s = time.perf_counter() - t0
            nu, npr = G.sizes()
            b = torch.zeros(nu + npr, dtype=torch.float64, device="cuda")
            b[:nu] = torch.as_tensor(np.random.default_rng(11).standard_normal(nu), device="cuda")
            r = torch.as_tensor(np.random.default_rng(1).standard_normal(nu + npr), device="cuda")
            z = torch.zeros_like(r)
            for _ in range(3):
                G.vcycle(r, z)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                G.vcycle(r, z)
            e1.record()
            torch.cuda.synchronize()
            vms = e0.elapsed_time(e1) / 10
            x = torch.zeros_like(b)
            st, _ = G.solve(b[:nu].contiguous(), b[nu:].contiguous(), x, tol=1e-8, maxit=400, check=False)
            rows.append(dict(n=n, degree=k, dofs=nu + npr, iterations=st.iterations, converged=bool(st.converged),
                             vcycle_ms=vms, dof_vcycles_per_s=(nu + npr) / (vms * 1e-3), solve_ms=st.solve_ms,
                             setup_s=setup_s))
            print(json.dumps(rows[-1]), flush=True)
            del G
            torch.cuda.empty_cache()
    print("\n| n | RT_k | dofs | iterations | V-cycle ms | DoF*V/s | solve ms |")
    for r_ in rows:
        print(f"| {r_['n']}^2 | RT_{r_['degree']} | {r_['dofs']:,} | {r_['iterations']} | {r_['vcycle_ms']:.2f} | "
              f"{r_['dof_vcycles_per_s']:.3g} | {r_['solve_ms']:.1f} |")
    return rows


def scale(torch, precision="fp32"):
    """Larger meshes and contrast 1e8 (NEXT-4): the driven flow of Tables 1-2
    on 2048^2 RT_0 cells (12.6 M dofs) and 512^2 RT_1 cells (3.1 M dofs),
    structures refined from 128^2, GMRES to a 1e-6 reduction."""
    rows = []
    for geom, case, model, mu, n, k in (("inclusions", "a", "Darcy", 0.0, 2048, 0),
                                        ("inclusions", "a", "Brinkman", 0.01, 2048, 0),
                                        ("connected", "b", "Brinkman", 0.01, 2048, 0),
                                        ("foam", "a", "Darcy", 0.0, 512, 1),
                                        ("connected", "a", "Brinkman", 0.01, 512, 1)):
        c = coefficient(geom, case, 1e8, n)
        t0 = time.perf_counter()
        st, x, G = driven_solve(torch, c, mu, degree=k, precision=precision)
        rows.append(dict(n=n, degree=k, geometry=geom, case=case, model=model, contrast=1e8,
                         dofs=int(x.numel()), iterations=st.iterations, converged=bool(st.converged),
                         solve_ms=st.solve_ms, setup_and_solve_s=time.perf_counter() - t0))
        print(json.dumps(rows[-1]), flush=True)
        del G, x
        torch.cuda.empty_cache()
    return rows


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="128,256,512")
    ap.add_argument("--contrasts", default="1e4,1e5,1e6")
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--coarse-avg", type=int, default=0, help="coarse coefficient: 0 arithmetic, 1 harmonic mean of c")
    ap.add_argument("--table4", action="store_true", help="the 3-D Brinkman analogue of Table 4 instead")
    ap.add_argument("--variants", action="store_true", help="smoother and cycle variants instead")
    ap.add_argument("--scale", action="store_true", help="2048^2 RT_0 and 512^2 RT_1 at contrast 1e8 instead")
    ap.add_argument("--degrees", action="store_true", help="RT_0, RT_1 and RT_2 on the same meshes instead")
    args = ap.parse_args()
    if args.degrees:
        degrees(torch, precision=args.precision)
        return
    if args.scale:
        scale(torch, precision=args.precision)
        return
    if args.table4:
        table4(torch, precision=args.precision)
        return
    if args.variants:
        variants(torch, precision=args.precision)
        return
    sizes = [int(s) for s in args.sizes.split(",")]
    contrasts = [float(s) for s in args.contrasts.split(",")]
    table = {}
    for case in ("a", "b"):
        for model, mu in (("Darcy", 0.0), ("Brinkman", 0.01)):
            for n in sizes:
                for geom in GEOMETRIES:
                    for kappa in contrasts:
                        c = coefficient(geom, case, kappa, n)
                        t0 = time.perf_counter()
                        st, _, G = driven_solve(torch, c, mu, precision=args.precision, coarse_avg=args.coarse_avg)
                        row = dict(case=case, model=model, n=n, geometry=geom, contrast=kappa,
                                   iterations=st.iterations, converged=bool(st.converged),
                                   rel_residual=st.rel_residual, solve_ms=st.solve_ms,
                                   wall_s=time.perf_counter() - t0)
                        print(json.dumps(row), flush=True)
                        table[(case, model, n, geom, kappa)] = st.iterations
                        del G
                        torch.cuda.empty_cache()
    for case in ("a", "b"):
        print(f"\ncase ({case}): GMRES iterations to a 1e-6 reduction")
        head = " | ".join(f"{g[:5]} {k:.0e}" for g in GEOMETRIES for k in contrasts)
        print(f"| model h^-1 | {head} |")
        for model in ("Darcy", "Brinkman"):
            for n in sizes:
                cells = " | ".join(str(table[(case, model, n, g, k)]) for g in GEOMETRIES for k in contrasts)
                print(f"| {model} {n} | {cells} |")


if __name__ == "__main__":
    main()
