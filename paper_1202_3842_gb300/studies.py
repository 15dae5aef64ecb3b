"""Scheme comparisons of the paper's Results section, run through the public API.

Each study builds its lattices with ``lbe.Simulation``, steps them on the GPU and returns plain
numbers; ``python -m paper_1202_3842_gb300.studies <study> [--quick]`` prints one JSON object.

- ``spurious``: the steady spurious current max|u|/v_T of a hard-sphere fluid at rest in the cosine
  well U = -eps (1 + cos(pi r / xi)) inside a periodic (4 xi)^3 box, for every scheme and several
  well sizes (Sec. "Results", the comparison of DD-TR with SD-TR and SD-EU).
- ``mixture``: the same for a binary mixture sigma 4/8 in FP32.
- ``stability``: the largest packing fraction at which each scheme runs a fixed number of steps in
  the well without a negative density (Sec. "Results", stability of TR against Euler).
- ``ideal_gas``: sigma = 0 in the cosine well: density error against the Boltzmann profile and the
  residual current, for the trapezoidal and the Euler integrator, against the well size (Sec. "Ideal
  fluid in a potential well").
- ``divergence``: max and mean |div u| in the bottleneck channel after a long run, per scheme.
- ``init``: the transient of the spurious current from the rest state and from the quasi-pressure
  state of the second distribution.
- ``visc``: stability with and without the viscous Enskog force.
- ``well_map``: stability of the method over packing and well depth at the production well's diameter
  and relaxation time (sigma 6, tau 0.8) on a 64^3 lattice.
- ``precision``: the storage precisions (FP32 and the shifted BF16 and FP16 forms) against FP64 on the
  128x32x32 bottleneck channel: density, velocity and time-averaged flux after the same steps.

Scheme names: ``dd_tr`` (the method, printed moment recovery), ``dd_tr_c`` (DD-TR with the
map-consistent recovery), ``sd_tr``, ``sd_eu``, ``dd_eu``.
"""
import argparse
import json
import math
import time

import numpy as np

from . import inputs, lbe

CS = math.sqrt(1.0 / 3.0)
SCHEMES = ("dd_tr", "dd_tr_c", "sd_tr", "sd_eu", "dd_eu")

# D3Q19 velocities and weights, for the host-side gradient used by the ideal-gas current shift.
_C = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
      (1, 1, 0), (1, -1, 0), (-1, 1, 0), (-1, -1, 0), (1, 0, 1), (1, 0, -1), (-1, 0, 1), (-1, 0, -1),
      (0, 1, 1), (0, 1, -1), (0, -1, 1), (0, -1, -1)]
_W = [1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12


def _split(scheme):
    """'dd_tr_c' -> ('dd_tr', True); other names pass through with the printed recovery."""
    if scheme not in SCHEMES:
        raise ValueError(f"unknown scheme {scheme!r}; expected one of {SCHEMES}")
    return (scheme[:-2], True) if scheme.endswith("_c") else (scheme, False)


def gradient_periodic(V, shape):
    """Isotropic lattice gradient 3 sum_p w_p c_p V(r + c_p) on a fully periodic lattice, [3][N].

    This is the discrete gradient that turns a potential into the force field F = -grad V."""
    nx, ny, nz = shape
    U = np.asarray(V, dtype=np.float64).reshape(nz, ny, nx)
    out = np.zeros((3, nz, ny, nx))
    for c, w in zip(_C, _W):
        if c == (0, 0, 0):
            continue
        shifted = np.roll(U, shift=(-c[2], -c[1], -c[0]), axis=(0, 1, 2))
        for a in range(3):
            if c[a]:
                out[a] += 3.0 * w * c[a] * shifted
    return out.reshape(3, -1)


def _well_sim(scheme, L, xi, sigmas, eta, prec, eps_kT=0.3, tau=1.0, check_every=200, n0=None):
    base, cons = _split(scheme)
    shape = (L, L, L)
    N = L ** 3
    sim = lbe.Simulation(shape, (1, 1, 1), len(sigmas), prec, scheme=base, consistent_moments=cons,
                         check_every=check_every)
    sim.set_geometry(np.zeros(N, np.uint8))
    V = inputs.cosine_well(shape, eps_kT, xi)
    # equal number densities; (pi/6) sum_a n sigma_a^3 = eta
    if n0 is None:
        n0 = 6.0 * eta / (math.pi * sum(s ** 3 for s in sigmas))
    for a, s in enumerate(sigmas):
        sim.set_species(a, s, tau)
        sim.set_potential(a, V)
        sim.set_body_force(a, (0.0, 0.0, 0.0))
    sim.set_wall_potential(np.zeros(N), np.zeros(N))
    for a in range(len(sigmas)):
        sim.init_density(a, np.full(N, n0))
    return sim, V, n0


def _run_current(sim, steps, chunk=500):
    """Step in chunks, recording max|u|/v_T after each; returns (ok, history or error text)."""
    hist = []
    try:
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            sim.step(k)
            done += k
            u = sim.velocity(-1)
            hist.append(float(np.sqrt((u ** 2).sum(0)).max() / CS))
        return True, hist
    except lbe.LbeError as e:
        return False, str(e)


def spurious(xis=(6, 9, 12, 16), schemes=SCHEMES, sigma=4.0, eta=0.2, steps=4000, prec="fp64"):
    """Steady spurious current per scheme and well size: {scheme: {xi: max|u|/v_T or None}}."""
    out = {}
    for s in schemes:
        out[s] = {}
        for xi in xis:
            sim, _, _ = _well_sim(s, 4 * xi, xi, [sigma], eta, prec)
            ok, hist = _run_current(sim, steps)
            sim.close()
            out[s][int(xi)] = dict(u=hist[-1], history=hist) if ok else dict(u=None, error=hist)
    return out


def mixture(schemes=SCHEMES, sigmas=(4.0, 8.0), eta=0.2, xi=12, steps=4000, prec="fp32"):
    """Spurious current of a binary mixture in the well: {scheme: {u, history} or {error}}."""
    out = {}
    for s in schemes:
        sim, _, _ = _well_sim(s, 4 * xi, xi, list(sigmas), eta, prec)
        ok, hist = _run_current(sim, steps)
        sim.close()
        out[s] = dict(u=hist[-1], history=hist) if ok else dict(u=None, error=hist)
    return out


def stability(schemes=SCHEMES, etas=(0.25, 0.27, 0.29, 0.31, 0.33, 0.37, 0.41), sigma=4.0, xi=8,
              steps=3000, prec="fp32"):
    """Largest stable packing per scheme: {scheme: {"stable": eta or None, "runs": {eta: ok}}}.

    Packings are tried in increasing order; the first divergence ends the scan of that scheme."""
    out = {}
    for s in schemes:
        runs, best = {}, None
        for eta in sorted(etas):
            sim, _, _ = _well_sim(s, 4 * xi, xi, [sigma], eta, prec)
            ok, _ = _run_current(sim, steps, chunk=steps)
            sim.close()
            runs[float(eta)] = ok
            if not ok:
                break
            best = float(eta)
        out[s] = dict(stable=best, runs=runs)
    return out


def ideal_gas(xis=(8, 12, 16, 24), schemes=("sd_tr", "sd_eu"), eps_kT=0.3, n0=0.01, steps_per_L2=3,
              prec="fp64"):
    """Resolution study of the ideal fluid in the cosine well.

    Runs steps_per_L2 * L^2 steps and reports Err(n) = max|n - n_eq| / n0 with the Boltzmann profile
    n_eq proportional to exp(-U / kT) at the same mean, Err(J) = max|J| / (n0 v_T) and the same for
    the shifted current J + n F / 2 (the Euler scheme's momentum is the plain sum over populations).
    Returns {scheme: {xi: {"n", "J", "J_shift"}}} and the log-log slopes between successive sizes."""
    out = {}
    for s in schemes:
        out[s] = {}
        for xi in xis:
            L = 4 * xi
            sim, V, _ = _well_sim(s, L, xi, [0.0], 0.0, prec, eps_kT=eps_kT, check_every=0, n0=n0)
            sim.step(steps_per_L2 * L * L)
            n = sim.density(0)
            J = sim.momentum(0)
            sim.close()
            F = -gradient_periodic(V, (L, L, L))
            neq = np.exp(-V / inputs.KT)
            neq *= n0 / neq.mean()
            Js = J + 0.5 * n[None, :] * F
            out[s][int(xi)] = dict(n=float(np.abs(n - neq).max() / n0),
                                   J=float(np.sqrt((J ** 2).sum(0)).max() / (n0 * CS)),
                                   J_shift=float(np.sqrt((Js ** 2).sum(0)).max() / (n0 * CS)))
    slopes = {}
    for s in schemes:
        xs = [int(x) for x in xis]
        slopes[s] = {k: [math.log(out[s][xs[i]][k] / out[s][xs[i + 1]][k]) / math.log(xs[i + 1] / xs[i])
                         for i in range(len(xs) - 1)] for k in ("n", "J", "J_shift")}
    return dict(errors=out, slopes=slopes)


def divergence(schemes=("dd_tr", "sd_tr", "sd_eu", "dd_eu"), shape=(128, 32, 32), width=16, length=64,
               body=1e-5, steps=20000, prec="fp64"):
    """|div u| of the barycentric velocity in the bottleneck channel after `steps` steps.

    Statistics are over interior fluid nodes (no blocked link, so the stencil does not straddle a
    wall).  Returns {scheme: {div_max, div_mean, u_max, flux} or {error}}."""
    out = {}
    for s in schemes:
        base, cons = _split(s)
        w = inputs.channel_workload(shape, (4.0, 6.0), 0.25, (1.0, 1.0), width, length, body=body)
        arr = inputs.build_workload(w)
        sim = lbe.Simulation(w["shape"], w["periodic"], 2, prec, scheme=base, consistent_moments=cons,
                             check_every=500)
        sim.set_geometry(arr["solid"])
        for a in range(2):
            sim.set_species(a, w["sigma"][a], w["tau"][a])
            sim.set_potential(a, arr["V"][a])
            sim.set_body_force(a, w["body"][a])
        for a in range(2):
            sim.init_density(a, arr["n"][a])
        sim.set_flux_plane(0, shape[0] // 2)
        try:
            sim.step(steps)
            d = sim.divergence(-1)
            u = sim.velocity(-1)
            inner = sim.link_mask() == 0
            fluid = arr["solid"] == 0
            out[s] = dict(div_max=float(np.abs(d[inner]).max()), div_mean=float(np.abs(d[inner]).mean()),
                          u_max=float(np.sqrt((u ** 2).sum(0))[fluid].max()), flux=float(sim.flux(-1)[1]))
        except lbe.LbeError as e:
            out[s] = dict(error=str(e))
        sim.close()
    return out


def init(xis=(6, 12), sigma=4.0, eta=0.2, steps=2000, prec="fp64", schemes=("dd_tr",)):
    """The transient from the two initial states of the second distribution: Pi(0) = n(0) (the default) and
    the quasi-pressure Pi = n - beta * path integral of C^mf + n F (Sec. "Stabilization").  Cosine well of
    size xi in a periodic (4 xi)^3 box, hard spheres at packing eta, uniform initial density; returns
    {scheme: {xi: {"rest": history, "quasipressure": history}}} of max|u|/v_T every 100 steps."""
    out = {}
    for s in schemes:
        out[s] = {}
        for xi in xis:
            res = {}
            for start in ("rest", "quasipressure"):
                sim, _, n0 = _well_sim(s, 4 * xi, xi, [sigma], eta, prec)
                if start == "quasipressure":
                    sim.init_density_quasipressure(np.full((1, (4 * xi) ** 3), n0))
                ok, hist = _run_current(sim, steps, chunk=100)
                sim.close()
                res[start] = hist if ok else {"error": hist}
            out[s][int(xi)] = res
    return out


def visc(cases=("well48", "channel128", "well24"), steps=600, prec="fp32", check=20):
    """Stability with and without the viscous Enskog force (an option of the DD-TR scheme): for each case
    the step at which a negative density appears (checked every `check` steps), or max|u|/v_T after
    `steps` steps.  Cases: "well48" (48^3, sigma 6, packing 0.3, Gaussian well 2 k_BT of radius 12,
    tau 0.8), "channel128" and "well24" (the named workloads of inputs.py), "well256"."""
    builders = {
        "well48": lambda: inputs.well_workload((48, 48, 48), 6.0, 0.3, 0.8, 2.0, 12.0),
        "channel128": inputs.WORKLOADS["channel128"],
        "well24": inputs.WORKLOADS["well24"],
        "well256": inputs.WORKLOADS["well256"],
    }
    out = {}
    for name in cases:
        w = builders[name]()
        arr = inputs.build_workload(w)
        M = len(w["sigma"])
        out[name] = {}
        for on in (False, True):
            sim = lbe.Simulation(w["shape"], w["periodic"], M, prec, visc=on, check_every=check)
            sim.set_geometry(arr["solid"])
            for a in range(M):
                sim.set_species(a, w["sigma"][a], w["tau"][a])
                sim.set_potential(a, arr["V"][a])
                sim.set_body_force(a, w["body"][a])
            sim.set_wall_potential(arr["phi"], arr["amp"])
            for a in range(M):
                sim.init_density(a, arr["n"][a])
            done = 0
            try:
                while done < steps:
                    sim.step(check)
                    done += check
                u = sim.velocity(-1)
                res = {"stable_steps": done, "u": float(np.sqrt((u ** 2).sum(0)).max() / CS)}
            except lbe.LbeError as e:
                res = {"diverged_by_step": done + check, "error": str(e)}
            finally:
                sim.close()
            out[name]["visc" if on else "plain"] = res
    return out


def well_map(etas=(0.1, 0.15, 0.2, 0.25, 0.3), depths=(0.5, 1.0, 2.0), L=64, radius=6.0, sigma=6.0, tau=0.8,
             steps=2000, check=50, prec="fp32"):
    """Stability of the DD-TR scheme (printed moment recovery) in the one-component Gaussian well at the
    diameter and relaxation time of the production-size well (sigma 6, tau 0.8), over packing and well
    depth, on a periodic L^3 lattice with the well radius scaled to the lattice (256^3 with radius 24
    becomes 64^3 with radius 6).  For each (packing, depth): the step by which a negative or non-finite
    density appeared (checked every `check` steps), or, for a run that lasts `steps`, max|u|/v_T and the
    density residual max|n(t) - n(t - check)| / (check n0) at the end."""
    out = {}
    for eta in etas:
        for depth in depths:
            w = inputs.well_workload((L, L, L), sigma, eta, tau, depth, radius)
            arr = inputs.build_workload(w)
            sim = lbe.Simulation(w["shape"], w["periodic"], 1, prec, check_every=check)
            res = {}
            try:
                sim.set_species(0, sigma, tau)
                sim.set_potential(0, arr["V"][0])
                sim.init_density(0, arr["n"][0])
                done = 0
                try:
                    while done < steps - check:
                        sim.step(check)
                        done += check
                    sim.residual()
                    sim.step(check)
                    done += check
                    r = sim.residual()
                    u = sim.velocity(-1)
                    res = {"stable_steps": done, "u": float(np.sqrt((u ** 2).sum(0)).max() / CS), "residual": r}
                except lbe.LbeError:
                    res = {"diverged_by_step": done + check}
            finally:
                sim.close()
            out["%g/%g" % (eta, depth)] = res
    return {"sigma": sigma, "tau": tau, "L": L, "radius": radius, "steps": steps, "runs": out}


def precision(steps=1000, precs=("fp64", "fp32", "bf16", "fp16"), workload="channel128", plane=None,
              keep_fields=False):
    """Each storage precision against the FP64 run of the same workload and step count (the FP64 path
    matches the FP64 oracle to 1e-12): for every precision, max over species and fluid nodes of
    |n - n64| / max n64 ("n"), |u^a - u^a_64| / max |u^a_64| ("u", per-species velocities J/n), and
    |flux - flux64| / |flux64| of the time-averaged plane flux, per species and summed ("flux",
    "flux_species").  The FP64 run's own values are returned under "reference"; keep_fields adds the
    fields of every run (n [M][N], J [M][3][N], time-averaged flux [M]) under "fields"."""
    w = inputs.WORKLOADS[workload]()
    arr = inputs.build_workload(w)
    M = len(w["sigma"])
    plane = w["shape"][0] // 2 if plane is None else plane
    fluid = arr["solid"] == 0
    runs = {}
    for prec in precs:
        sim = lbe.Simulation(w["shape"], w["periodic"], M, prec)
        try:
            sim.set_geometry(arr["solid"])
            for a in range(M):
                sim.set_species(a, w["sigma"][a], w["tau"][a])
                sim.set_potential(a, arr["V"][a])
                sim.set_body_force(a, w["body"][a])
            for a in range(M):
                sim.init_density(a, arr["n"][a])
            sim.set_flux_plane(0, plane)
            sim.step(steps)
            runs[prec] = {"n": [sim.density(a) for a in range(M)], "u": [sim.velocity(a) for a in range(M)],
                          "flux": [sim.flux(a)[1] for a in range(M)]}
            if keep_fields:
                runs[prec]["J"] = [sim.momentum(a) for a in range(M)]
        finally:
            sim.close()
    ref = runs["fp64"]
    out = {"workload": workload, "steps": steps, "flux_plane_x": plane,
           "reference": {"flux_species": ref["flux"], "max_n": [float(ref["n"][a].max()) for a in range(M)],
                         "max_u": [float(np.abs(ref["u"][a][:, fluid]).max()) for a in range(M)]}}
    ftot = sum(ref["flux"])
    for prec, r in runs.items():
        out[prec] = {
            "n": max(float(np.abs(r["n"][a] - ref["n"][a])[fluid].max() / ref["n"][a].max()) for a in range(M)),
            "u": max(float(np.abs(r["u"][a] - ref["u"][a])[:, fluid].max() / np.abs(ref["u"][a][:, fluid]).max())
                     for a in range(M)),
            "flux_species": [abs(r["flux"][a] - ref["flux"][a]) / abs(ref["flux"][a]) for a in range(M)],
            "flux": abs(sum(r["flux"]) - ftot) / abs(ftot)}
    if keep_fields:
        out["fields"] = {prec: {k: r[k] for k in ("n", "J", "flux")} for prec, r in runs.items()}
    return out


# Reduced sizes for a quick look (a few seconds each on one GPU).
QUICK = {
    "spurious": dict(xis=(6,), steps=1000),
    "mixture": dict(xi=6, steps=1000),
    "stability": dict(etas=(0.25, 0.29), steps=500),
    "ideal_gas": dict(xis=(4, 6), steps_per_L2=3),
    "divergence": dict(shape=(64, 32, 32), length=32, steps=1000),
    "init": dict(xis=(6,), steps=500),
    "visc": dict(cases=("well48", "well24"), steps=200),
    "precision": dict(steps=200),
    "well_map": dict(etas=(0.1, 0.3), depths=(0.5, 2.0), L=32, radius=3.0, steps=300),
}
STUDIES = dict(spurious=spurious, mixture=mixture, stability=stability, ideal_gas=ideal_gas,
               divergence=divergence, init=init, visc=visc, precision=precision, well_map=well_map)


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("study", choices=sorted(STUDIES))
    p.add_argument("--quick", action="store_true", help="reduced sizes and step counts")
    p.add_argument("--schemes", default=None, help="comma-separated subset of " + ",".join(SCHEMES))
    args = p.parse_args(argv)
    kw = dict(QUICK[args.study]) if args.quick else {}
    if args.schemes:
        kw["schemes"] = tuple(args.schemes.split(","))
        for s in kw["schemes"]:
            _split(s)
    t0 = time.time()
    res = STUDIES[args.study](**kw)
    print(json.dumps(dict(study=args.study, quick=args.quick, seconds=round(time.time() - t0, 1),
                          result=res)))


if __name__ == "__main__":
    main()
