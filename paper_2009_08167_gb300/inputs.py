"""Seeded synthetic inputs shared by the tests, the bench and the smoke run.

This module holds no arithmetic of the eigensolution: it only describes
meshes (elements per side, degree, interior knot multiplicities) and draws
random numbers.  Random numbers come from SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): state +=
0x9E3779B97F4A7C15, then two xor-shift-multiply rounds.  Normal deviates use
the Box-Muller transform on pairs of 53-bit uniforms in (0, 1].
"""
import numpy as np

_MASK = (1 << 64) - 1


def splitmix64(seed, n):
    """n successive SplitMix64 outputs (uint64) from ``seed``."""
    out = np.empty(n, dtype=np.uint64)
    s = int(seed) & _MASK
    for i in range(n):
        s = (s + 0x9E3779B97F4A7C15) & _MASK
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out[i] = z ^ (z >> 31)
    return out


def uniform01(seed, n):
    """Uniforms in (0, 1]: (top 53 bits + 1) / 2^53."""
    u = splitmix64(seed, n)
    return ((u >> np.uint64(11)).astype(np.float64) + 1.0) / 9007199254740992.0


def normal(seed, n, std=1.0):
    """n N(0, std^2) deviates by Box-Muller."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * np.pi * u[1::2]
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(t)
    z[1::2] = r * np.sin(t)
    return std * z[:n]


def separator_multiplicities(ne, p, bs):
    """Interior knot multiplicities for blocks of ``bs`` elements: p at every
    bs-th interior knot (a C0 separator line), 1 elsewhere; bs >= ne is the
    maximum-continuity mesh."""
    return [p if (0 < bs < ne and i % bs == 0) else 1 for i in range(1, ne)]


class Mesh:
    """Tensor-product mesh on [0,1]^dim: elements per side, degree, interior
    knot multiplicities per direction, leaf extent of the dissection."""

    def __init__(self, dim, ne, p, bs=None, leaf_extent=8):
        self.dim = dim
        self.ne = [ne] * dim if np.isscalar(ne) else list(ne)
        self.p = p
        self.bs = bs
        self.leaf_extent = leaf_extent
        if bs is None:
            self.mults = [[1] * (n - 1) for n in self.ne]
        else:
            self.mults = [separator_multiplicities(n, p, bs) for n in self.ne]

    @property
    def n_elem(self):
        return int(np.prod(self.ne))

    def __repr__(self):
        return f"Mesh(dim={self.dim}, ne={self.ne}, p={self.p}, bs={self.bs}, leaf_extent={self.leaf_extent})"


def config_c1():
    """2D, p=2, 16x16 elements, maximum continuity, sigma=0, 10 pairs."""
    return dict(mesh=Mesh(2, 16, 2, None), k=10, sigma=0.0)


def config_c2(riga=True):
    """2D, p=3, 256x256 elements; rIGA with C0 lines every 16 elements (or
    maximum continuity); 100 pairs in two slices of 50."""
    return dict(mesh=Mesh(2, 256, 3, 16 if riga else None), k=100, sigma=0.0, slice=50)


def config_c3():
    """3D, p=2, 64^3 elements, C0 planes every 8 elements, 50 pairs."""
    return dict(mesh=Mesh(3, 64, 2, 8), k=50, sigma=0.0)


def config_c5(seed=0xC5):
    """2D rIGA p=3, 128x128, C0 lines every 16 elements, coefficients
    exp(a_e), exp(b_e) with a_e, b_e ~ N(0, 0.25^2); 20 pairs."""
    mesh = Mesh(2, 128, 3, 16)
    z = normal(seed, 2 * mesh.n_elem, 0.25)
    return dict(mesh=mesh, a=z[:mesh.n_elem], b=z[mesh.n_elem:], k=20, sigma=0.0)


def config_c4(n_problems=512, seed=0xC4):
    """Batch of 2D rIGA problems: elements per side U{32..128}, p in {2,3},
    block size in {8,16}, a_e ~ N(0, 0.5^2) per element; 20 pairs each."""
    u = splitmix64(seed, 3 * n_problems)
    probs = []
    for i in range(n_problems):
        ne = 32 + int(u[3 * i] % np.uint64(97))
        p = 2 + int(u[3 * i + 1] % np.uint64(2))
        bs = 8 if int(u[3 * i + 2] % np.uint64(2)) == 0 else 16
        mesh = Mesh(2, ne, p, bs)
        a = normal(seed * 1000003 + i, mesh.n_elem, 0.5)
        probs.append(dict(mesh=mesh, a=a, k=20, sigma=0.0))
    return probs
