"""Method fidelity of the coupled ROM against fine grids (test
infrastructure, like the rest of the oracle): the comparison of section
"Numerical experiments", where the ROM's traces are measured against a
reference fine-grid solution by their relative L2 error.

Three runs of the same problem, all FP64 leapfrog at 0.9 of their own
stability limit, over [0, t_end]:

* the global fine grid (every node shared across subdomain boundaries);
* the "slit" fine grid, in which only open-face nodes are shared (the limit
  the ROM converges to under the open-face reading of the face basis);
* the coupled ROM (Algorithm 1), its traces interpolated linearly in time
  onto the fine grid's samples (its step is larger).

Each starts either from rest with the problem's Ricker point source, or
from a Gaussian initial displacement at the source position (Algorithm 1's
own form: initial conditions projected by Eq. 16, no source term).

``python -m oracle.fidelity --cells-per-unit 20 --m 25 --k 3`` prints one
JSON line for the stand-in of the paper's 7 x 7 x 3 layout."""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

import sfm_inputs as inputs

from . import coupled, fine, pipeline


def trace_errors(problem, t_end, u0=None):
    """Relative L2 trace errors (all receivers and samples) of the ROM
    against the global and the slit fine grids, and of the slit grid against
    the global one; plus the time steps and the ROM's size.  With ``u0`` (a
    nodal field [nz+1, ny+1, nx+1]) every run starts from that displacement
    at rest and the point source is silent; otherwise the runs start from
    rest and the source emits the problem's Ricker wavelet."""
    if u0 is None:
        ws = lambda dt, n: inputs.ricker(np.arange(n) * dt, problem.f_peak)[None]
    else:
        ws = lambda dt, n: np.zeros((1, n))
    t0 = time.time()
    fs = pipeline.fine_system(problem)
    dtf = 0.9 * fine.cfl_dt(fs[0], fs[1])
    nf = int(np.ceil(t_end / dtf))
    dtf = t_end / nf
    ref = pipeline.fine_traces(fs, dtf, nf, ws(dtf, nf),
                               None if u0 is None else np.asarray(u0, np.float64).ravel())
    del fs
    ss = pipeline.slit_system(problem)
    slit = pipeline.fine_traces(ss, dtf, nf, ws(dtf, nf),
                                None if u0 is None else pipeline.slit_field(problem, u0))
    del ss
    rs = pipeline.build(problem, u0=u0)
    dt = pipeline.rom_dt(rs)
    n = int(np.ceil(t_end / dt))
    dt = t_end / n
    d = coupled.step_structured(rs, dt, n, ws(dt, n), U0=None if u0 is None else rs.U0)
    tf = np.arange(nf + 1) * dtf
    tr = np.arange(n + 1) * dt
    di = np.stack([[np.interp(tf, tr, d[q, r]) for r in range(d.shape[1])]
                   for q in range(d.shape[0])])
    return {
        "rom_vs_fine": pipeline.rel_l2(di, ref),
        "rom_vs_slit": pipeline.rel_l2(di, slit),
        "slit_vs_fine": pipeline.rel_l2(slit, ref),
        "dt_fine": dtf, "dt_rom": dt, "steps_fine": nf, "steps_rom": n,
        "rom_dof": int(np.sum(rs.k * rs.b)),
        "fine_nodes": int((problem.nx + 1) * (problem.ny + 1) * (problem.nz + 1)),
        "seconds": time.time() - t0,
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--cells-per-unit", type=int, default=20)
    ap.add_argument("--m", type=int, default=25)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--sigma-factor", type=float, default=None,
                    help="shift (2 pi factor f_peak)^2 instead of the layout's")
    ap.add_argument("--shift-factors", default=None,
                    help="comma-separated factors f_j of distinct shifts (2 pi f_j f_peak)^2, "
                         "one per block after the first (Eq. 6)")
    ap.add_argument("--source-x", type=float, default=None)
    ap.add_argument("--start", choices=("source", "pulse"), default="source",
                    help="a Ricker point source from rest, or a Gaussian initial pulse "
                         "at the source position")
    a = ap.parse_args(argv)
    p = inputs.paper_layout(cells_per_unit=a.cells_per_unit, m=a.m, k=a.k)
    if a.sigma_factor is not None:
        p.sigma = inputs.default_sigma(p.f_peak, a.sigma_factor)
    if a.shift_factors:
        p.sigma = [inputs.default_sigma(p.f_peak, float(f)) for f in a.shift_factors.split(",")]
    if a.source_x is not None:
        p.src_xyz[0, 0] = a.source_x
    u0 = None
    if a.start == "pulse":
        u0 = inputs.gaussian_pulse(p, p.src_xyz[0], 3.0 * 0.78 / (2.0 * np.pi))
    out = {"workload": p.name, "cells_per_unit": a.cells_per_unit, "m": a.m, "k": a.k,
           "sigma": p.sigma if np.ndim(p.sigma) else float(p.sigma),
           "source": p.src_xyz[0].tolist(), "start": a.start}
    out.update(trace_errors(p, p.meta["t_end"], u0))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
