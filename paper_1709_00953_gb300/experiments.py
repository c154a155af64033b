"""Re-runs of the paper's 2D studies of Sec. III on a seeded phantom, on the GPU.

The set-up follows Sec. III: a 64 x 64 image of unit pixels; a flat detector
of 187 unit pixels kept perpendicular to the central ray; source and detector
centre on circles of radius 115 about the image centre (SOD 115, SDD 230);
360 views 1 degree apart.  The image is split into t x t volume blocks (J) and
every view's detector into k sub-areas; a row block (I) is one sub-area of one
view, so there are 360 k row blocks, drawn by density (importance sampling)
unless a study says otherwise.

Data are consistent and noise-free, y = A x_true, for a seeded random-ellipse
phantom (the paper's phantom is not available, so the studies show trends, not
the printed SNRs).  Quality after each epoch is the paper's
SNR = 20 log10 |x_true| / |x_true - x| and the observation gap
20 log10 |y| / |y - A x|, against effective epochs = epochs x alpha.

Studies (each a list of runs over one parameter):
  beta   - b in {70, 100, 130, 160, 190} (the paper's range) and 400 .. 4000
           (where it breaks down here), alpha = 1, group size 1 (Sec. III-A)
  alpha  - alpha in {1, 0.8, 0.5, 0.2}, b = 100, group size 1 (Sec. III-B)
  group  - (group size, b) in {(1, 100), (5, 25), (100, 2)}, alpha = 0.5 (Sec. III-B)
  det    - 2, 4, 8, 16 detector sub-areas, group size 1 with b = 50 k and group
           size 100 with b = k (Sec. III-C)
  vol    - 2, 4, 8, 16 blocks per image axis, group size 100, b = 4 / t (Sec. III-C)
  gamma  - gamma in {1, 0.75, 0.5, 0.25} with 4 x 4 blocks (b = 1) and 8 x 8
           blocks (b = 0.5), group size 100 (Sec. III-C)
  sampling - importance, uniform and mixed (theta step 1/40) sampling for group
           sizes 1, 5, 100 (b = 100, 25, 2), alpha = 0.5, three schedule seeds
           each (Sec. III-D)
  3d     - the 3D scan of Sec. III-E (Problem3D): group size 90, b = 1,
           alpha = 0.5, 200 effective epochs

Run as ``python -m paper_1709_00953_gb300.experiments [study ...]``: prints one
JSON object per run.
"""
from __future__ import annotations

import json
import math
import sys

import numpy as np

from . import csgd

N = 64
SOD = 115.0
SDD = 230.0
N_DET = 187
N_VIEWS = 360
PHANTOM_SHAPES = 10
PHANTOM_SEED = 1709 + 30
SCHEDULE_SEED = 0x17090953 + 30


def geometry_spec() -> dict:
    return dict(kind="fan2d_flat", n=(N, N), h=1.0,
                angles=np.deg2rad(np.arange(N_VIEWS, dtype=np.float64)), nu=N_DET, nv=1,
                pu=1.0, pv=1.0, sod=SOD, sdd=SDD)


def phantom_image() -> np.ndarray:
    """x_true: pixel averages of a seeded random-ellipse phantom, x fastest."""
    from synth import phantom as PH
    ph = PH.make_phantom(2, PHANTOM_SHAPES, 0.5 * N, PHANTOM_SEED)
    return PH.pixelize(ph, (N, N), 1.0).astype(np.float32)


def groups_per_epoch(flat: list, n_epochs: int) -> list:
    """Group steps of each epoch in the flat schedule encoding of
    csgd_schedule_generate (per epoch: n_cols, then per column: j, n_groups,
    then per group: size, rows...)."""
    out, k = [], 0
    for _ in range(n_epochs):
        ncols = flat[k]
        k += 1
        cnt = 0
        for _ in range(ncols):
            ng = flat[k + 1]
            k += 2
            for _ in range(ng):
                k += 1 + flat[k]
                cnt += 1
        out.append(cnt)
    return out


class Problem:
    """One partition of the Sec. III scan with its consistent data on the GPU."""

    def __init__(self, tiles: int = 2, det_parts: int = 2):
        import torch
        self.torch = torch
        self.geom = csgd.Geometry(geometry_spec())
        self.part = csgd.Partition(self.geom, tiles=(tiles, tiles), view_blocks=N_VIEWS,
                                   det_blocks=(det_parts, 1))
        self.x_true = torch.tensor(phantom_image(), device="cuda")
        self.y = torch.zeros(self.part.n_rays, dtype=torch.float32, device="cuda")
        csgd.project_full(self.part, self.x_true, self.y)
        torch.cuda.synchronize()
        self.y_norm = float(torch.linalg.vector_norm(self.y.double()))
        self.x_norm = float(torch.linalg.vector_norm(self.x_true.double()))

    def run(self, b: float, alpha: float = 1.0, group_size: int = 1, gamma: float = 1.0,
            eff_epochs: float = 50.0, sampling: int = csgd.IMPORTANCE,
            seed: int = SCHEDULE_SEED) -> dict:
        """CSGD / GCSGD (Alg. 3 / Alg. 4) from x = 0; SNR and observation gap
        after every epoch up to eff_epochs effective epochs."""
        return run_solver(self, b, alpha, group_size, gamma, eff_epochs, sampling, seed)


def run_solver(p, b, alpha, group_size, gamma, eff_epochs, sampling, seed) -> dict:
    """The solve loop of every study: p holds the partition, the data y, x_true
    and their norms.  Records SNR and observation gap after every epoch."""
    import torch
    params = dict(sampling=sampling, alpha=alpha, gamma=gamma, b=b, group_size=group_size,
                  seed=seed)
    n_epochs = max(1, int(round(eff_epochs / alpha)))
    steps = groups_per_epoch(csgd.schedule_generate(p.part, params, n_epochs), n_epochs)
    solver = csgd.Solver(p.part, params, p.y)
    x = torch.zeros(p.part.n_voxels, dtype=torch.float32, device="cuda")
    snr, gap, epochs = [], [], []
    for e in range(n_epochs):
        rep = solver.solve(steps[e], x, residual=True)
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm((p.x_true - x).double()))
        snr.append(20.0 * math.log10(p.x_norm / err) if err > 0 else math.inf)
        res = rep["residual_norm"]
        gap.append(20.0 * math.log10(p.y_norm / res) if res > 0 else math.inf)
        epochs.append(rep["epochs"])
    return dict(b=b, alpha=alpha, group_size=group_size, gamma=gamma, sampling=sampling,
                seed=seed, eff_epochs=[(e + 1) * alpha for e in range(n_epochs)],
                epochs=epochs, steps_per_epoch=steps, snr_db=snr, gap_db=gap,
                x=x.cpu().numpy())


class Problem3D:
    """The 3D scan of Sec. III-E: 128^3 voxels over a 32^3 volume (h = 0.25),
    720 views on a random spherical trajectory of radius 66 about the volume's
    centre, a flat square detector perpendicular to the source-centre line at
    distance 132 with 202 x 202 pixels at pitch 0.5 (the paper's side length
    101 read as a length), each view one row block, 2 x 2 x 2 volume blocks;
    consistent data y = A x_true of a seeded random-ellipsoid phantom."""

    def __init__(self, n: int = 128, views: int = 720, pixels: int = 202):
        import torch
        from synth import configs as C
        from synth import phantom as PH
        self.torch = torch
        h = 32.0 / n
        spec = dict(kind="custom3d", n=(n, n, n), h=h, nu=pixels, nv=pixels, pu=0.5, pv=0.5,
                    poses=C.random_sphere_poses(views, 66.0, 132.0, seed=PHANTOM_SEED + 3))
        self.geom = csgd.Geometry(spec)
        self.part = csgd.Partition(self.geom, tiles=(2, 2, 2), view_blocks=views)
        ph = PH.make_phantom(3, 10, 16.0, PHANTOM_SEED + 3)
        self.x_true = PH.pixelize(ph, (n, n, n), h, sub=2, xp=torch, device="cuda").float()
        self.y = torch.zeros(self.part.n_rays, dtype=torch.float32, device="cuda")
        csgd.project_full(self.part, self.x_true, self.y)
        torch.cuda.synchronize()
        self.y_norm = float(torch.linalg.vector_norm(self.y.double()))
        self.x_norm = float(torch.linalg.vector_norm(self.x_true.double()))

    def run(self, b: float = 1.0, alpha: float = 0.5, group_size: int = 90, gamma: float = 1.0,
            eff_epochs: float = 200.0, sampling: int = csgd.IMPORTANCE,
            seed: int = SCHEDULE_SEED) -> dict:
        return run_solver(self, b, alpha, group_size, gamma, eff_epochs, sampling, seed)


def study(name: str, eff_epochs: float = 50.0) -> list:
    """The runs of one study (see the module docstring); each run's dict gains
    the partition it used."""
    runs, problems = [], {}

    def go(tiles, det, **kw):
        if (tiles, det) not in problems:
            problems[(tiles, det)] = Problem(tiles, det)
        r = problems[(tiles, det)].run(eff_epochs=eff_epochs, **kw)
        r.update(study=name, tiles=tiles, det_parts=det)
        runs.append(r)

    if name == "beta":
        for b in (70.0, 100.0, 130.0, 160.0, 190.0, 400.0, 1000.0, 2000.0, 4000.0):
            go(2, 2, b=b, alpha=1.0, group_size=1)
    elif name == "alpha":
        for a in (1.0, 0.8, 0.5, 0.2):
            go(2, 2, b=100.0, alpha=a, group_size=1)
    elif name == "group":
        for s, b in ((1, 100.0), (5, 25.0), (100, 2.0)):
            go(2, 2, b=b, alpha=0.5, group_size=s)
    elif name == "det":
        for k in (2, 4, 8, 16):
            go(2, k, b=50.0 * k, alpha=0.5, group_size=1)
            go(2, k, b=float(k), alpha=0.5, group_size=100)
    elif name == "vol":
        for t in (2, 4, 8, 16):
            go(t, 2, b=4.0 / t, alpha=0.5, group_size=100)
    elif name == "gamma":
        for t, b in ((4, 1.0), (8, 0.5)):
            for g in (1.0, 0.75, 0.5, 0.25):
                go(t, 2, b=b, alpha=0.5, group_size=100, gamma=g)
    elif name == "sampling":
        for s, b in ((1, 100.0), (5, 25.0), (100, 2.0)):
            for sampling in (csgd.IMPORTANCE, csgd.UNIFORM, csgd.MIXED):
                for rep in range(3):
                    go(2, 2, b=b, alpha=0.5, group_size=s, sampling=sampling,
                       seed=SCHEDULE_SEED + rep)
    elif name == "3d":
        r = Problem3D().run(eff_epochs=eff_epochs)
        r.update(study=name, tiles=2, det_parts=1)
        runs.append(r)
    else:
        raise ValueError("unknown study %r" % name)
    return runs


STUDIES = ("beta", "alpha", "group", "det", "vol", "gamma", "sampling", "3d")


def main(argv=None) -> None:
    names = (argv if argv else list(STUDIES))
    from . import build
    build.build()
    for name in names:
        for r in study(name, eff_epochs=200.0 if name == "3d" else 50.0):
            r = dict(r)
            r.pop("x")
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
