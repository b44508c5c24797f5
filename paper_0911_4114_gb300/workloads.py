"""Seeded synthetic inputs shaped like the paper's and the benchmark's workloads.

Only random numbers live here (numpy PCG64, seed = 20260000 + workload index); none of
the method's arithmetic.  Shared by the tests, bench.py and the oracle runs.
"""
import numpy as np

SEED0 = 20260000


def rng(index, salt=0):
    return np.random.Generator(np.random.PCG64(SEED0 + index + 1000 * salt))


def cube(n, g):
    """n points i.i.d. uniform in [0, 1]^3 (Section 3.5.3 uses a uniform cube)."""
    return g.random((n, 3))


def sphere(n, g, radius=1.0):
    """n points uniform on a sphere: normalised i.i.d. N(0,1) 3-vectors."""
    p = g.standard_normal((n, 3))
    return radius * p / np.linalg.norm(p, axis=1)[:, None]


def ellipsoid(n, g, axes=(1.0, 0.5, 0.25)):
    """n points uniform by area on an ellipsoid surface (accept-reject on the unit sphere)."""
    a, b, c = axes
    gmax = max(a * b, a * c, b * c)
    out = np.empty((0, 3))
    while out.shape[0] < n:
        u = sphere(2 * (n - out.shape[0]) + 64, g)
        gg = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
        keep = g.random(u.shape[0]) < gg / gmax
        out = np.concatenate([out, u[keep] * np.array(axes)])
    return out[:n]


def clusters(n, g, nclusters=16, background=0.1):
    """Strongly clustered cloud in [0, 1]^3: a fraction `background` uniform in the cube, the
    rest split evenly over `nclusters` small cubes (sides uniform in [0.02, 0.08], centres
    uniform in [0.1, 0.9]^3): densities differ by three to four orders of magnitude."""
    nb = int(round(background * n))
    parts = [cube(nb, g)]
    sizes = np.full(nclusters, (n - nb) // nclusters)
    sizes[: (n - nb) - int(sizes.sum())] += 1
    for m in sizes:
        c = g.uniform(0.1, 0.9, 3)
        h = g.uniform(0.02, 0.08)
        parts.append(c + h * (g.random((int(m), 3)) - 0.5))
    return np.concatenate(parts)


def charges(n, nrhs, g):
    """complex charges, re and im i.i.d. N(0,1), shape (n, nrhs) (or (n,) for nrhs=0)."""
    shape = (n,) if nrhs == 0 else (n, nrhs)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


# named workloads: (index, description)
WORKLOADS = {
    "cube4k_fp64": 0,       # 4,096 uniform in [0,1]^3, kappa 8 pi, eps 1e-6, depth 3
    "sphere262k": 1,        # 262,144 on the unit sphere, kappa 64, eps 1e-6
    "ellipsoid2m": 2,       # 2,097,152 on the (1, .5, .25) ellipsoid, kappa 200
    "cube512k_rhs64": 3,    # 524,288 uniform cube, kappa 40, 64 RHS, eps 1e-5
    "spheres131k_grad": 4,  # 131,072 on r=1 (sources) and r=1.5 (targets), kappa 32
    "clusters1m": 5,        # 1,048,576 in 16 dense small cubes + 10% uniform, kappa 72.5
}


def points(name, n=None):
    i = WORKLOADS[name]
    g = rng(i)
    if name == "cube4k_fp64":
        x = cube(n or 4096, g)
        return x, x
    if name == "sphere262k":
        x = sphere(n or 262144, g)
        return x, x
    if name == "ellipsoid2m":
        x = ellipsoid(n or 2097152, g)
        return x, x
    if name == "cube512k_rhs64":
        x = cube(n or 524288, g)
        return x, x
    if name == "clusters1m":
        x = clusters(n or 1048576, g)
        return x, x
    if name == "spheres131k_grad":
        s = sphere(n or 131072, g)
        t = sphere(n or 131072, g, radius=1.5)
        return s, t
    raise KeyError(name)
