"""Independent closed forms used to pin the oracle (test helpers, not the oracle).

- fully discrete Fourier solution of the central-difference / RK2 scheme;
- exact characteristic solution of constant-coefficient advection;
- projector-product form of the root-to-leaves HSVD built from full-matrix SVDs.
"""
import numpy as np


def fourier_rk2(u0: np.ndarray, c, h: float, dt: float, steps: int) -> np.ndarray:
    """u_n = IFFT[ R(dt*lam)^n FFT(u0) ], lam(k) = -i sum_j c_j sin(k_j h)/h, R = 1+z+z^2/2.

    The periodic central difference maps e^{i k x} to (i sin(k h)/h) e^{i k x}.
    """
    uh = np.fft.fftn(u0)
    lam = np.zeros(u0.shape, dtype=np.complex128)
    for j, n in enumerate(u0.shape):
        k = np.fft.fftfreq(n) * n
        s = np.sin(k * h) / h
        shape = [1] * u0.ndim
        shape[j] = n
        lam = lam + (-1j * c[j] * s).reshape(shape)
    z = dt * lam
    R = 1.0 + z + 0.5 * z * z
    return np.fft.ifftn(uh * R ** steps).real


def fourier_ab2(u0: np.ndarray, u1: np.ndarray, c, h: float, dt: float, steps: int) -> np.ndarray:
    """AB2 on every Fourier mode: w_{n+1} = (1 + 3z/2) w_n - (z/2) w_{n-1}, z = dt lam(k), from
    the two start levels u0, u1; returns the level `steps` after u1."""
    lam = np.zeros(u0.shape, dtype=np.complex128)
    for j, n in enumerate(u0.shape):
        k = np.fft.fftfreq(n) * n
        shape = [1] * u0.ndim
        shape[j] = n
        lam = lam + (-1j * c[j] * np.sin(k * h) / h).reshape(shape)
    z = dt * lam
    a, b = np.fft.fftn(u0), np.fft.fftn(u1)
    for _ in range(steps):
        a, b = b, (1.0 + 1.5 * z) * b - 0.5 * z * a
    return np.fft.ifftn(b).real


def matricize(full: np.ndarray, dims: list) -> np.ndarray:
    rest = [i for i in range(full.ndim) if i not in dims]
    nr = int(np.prod([full.shape[i] for i in dims]))
    return full.transpose(dims + rest).reshape(nr, -1, order="F")


def apply_node_projector(full: np.ndarray, dims: list, P: np.ndarray) -> np.ndarray:
    """Apply P (N_t x N_t) to the node matricisation rows and fold back."""
    rest = [i for i in range(full.ndim) if i not in dims]
    perm = dims + rest
    shp = [full.shape[i] for i in perm]
    M = matricize(full, dims)
    Y = (P @ M).reshape(shp, order="F")
    inv = np.argsort(perm)
    return Y.transpose(inv)


def varcoef_L_shifted_gaussian(zs: list, C: np.ndarray, mu) -> np.ndarray:
    """-sum_j (C z)_j d/dz_j applied to g(z) = exp(-|z - mu|^2) on the full grid of the 1-D
    grids zs: d g / dz_j = -2 (z_j - mu_j) g, so L g = 2 g sum_j (C z)_j (z_j - mu_j)."""
    Zs = np.meshgrid(*zs, indexing="ij")
    g = np.exp(-sum((Z - m) ** 2 for Z, m in zip(Zs, mu)))
    N = len(zs)
    out = np.zeros_like(g)
    for j in range(N):
        a = sum(C[j, k] * Zs[k] for k in range(N))
        out += a * (Zs[j] - mu[j])
    return 2.0 * g * out


def varcoef_exact(t: float, C: np.ndarray, z) -> float:
    """Characteristic solution f(z, t) = f0(exp(-tC) z) with f0 = exp(-|z|^2) (Section 4.1)."""
    from scipy.linalg import expm
    y = expm(-t * C) @ np.asarray(z, dtype=np.float64)
    return float(np.exp(-(y @ y)))
