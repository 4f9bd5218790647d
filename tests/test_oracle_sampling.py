"""Pins for the oracle's FP32 sampling routines against mathematics they must reproduce:
library sine/cosine, the cosine-weighted distribution, the GGX directional albedo by
quadrature of the microfacet BRDF, and orthonormal tangent frames."""
import math

import numpy as np
import pytest


def _ulp_err(got, exact):
    got = np.float32(got)
    exact32 = np.float32(exact)
    ulp = np.spacing(np.abs(exact32)).astype(np.float64)
    ulp = np.where(ulp == 0, np.spacing(np.float32(1e-38)), ulp)
    return abs(float(got) - exact) / ulp


def test_sincos_within_2ulp(orc):
    xs = np.linspace(-math.pi / 4, math.pi / 4, 20001).astype(np.float32)
    xs = np.concatenate([xs, np.float32([0.0, 1e-8, -1e-8, 1e-3, np.float32(math.pi / 4)])])
    worst_s = worst_c = 0.0
    for x in xs:
        s, c = orc.sincos(x)
        worst_s = max(worst_s, _ulp_err(s, math.sin(float(x))))
        worst_c = max(worst_c, _ulp_err(c, math.cos(float(x))))
    assert worst_s <= 2.0 and worst_c <= 2.0, (worst_s, worst_c)


def _stratified(n):
    g = (np.arange(n) + 0.5) / n
    u1, u2 = np.meshgrid(g, g, indexing="ij")
    return np.float32(u1.ravel()), np.float32(u2.ravel())


def test_cosine_sampling_distribution(orc):
    """Cosine-weighted hemisphere: z^2 is uniform on [0,1], azimuth uniform, E[z] = 2/3."""
    u1, u2 = _stratified(128)
    w = np.array([orc.sample_cosine(a, b) for a, b in zip(u1, u2)], dtype=np.float64)
    rng = np.random.default_rng(5)
    r = rng.random((20000, 2)).astype(np.float32)
    assert (w[:, 2] >= 0).all()
    assert np.abs(np.linalg.norm(w, axis=1) - 1).max() < 1e-6
    assert abs(w[:, 2].mean() - 2 / 3) < 1e-3  # uniform-hemisphere would give 1/2
    # Kolmogorov-Smirnov on random (not stratified) uniforms: z^2 ~ U(0, 1)
    z2 = np.sort(np.array([orc.sample_cosine(a, b)[2] for a, b in r], dtype=np.float64) ** 2)
    ks = np.abs(z2 - (np.arange(z2.size) + 0.5) / z2.size).max()
    assert ks < 1.95 / np.sqrt(z2.size)  # p ~ 1e-3
    wr = np.array([orc.sample_cosine(a, b) for a, b in r[:8000]], dtype=np.float64)
    hist, _ = np.histogram(np.arctan2(wr[:, 1], wr[:, 0]), bins=16, range=(-np.pi, np.pi))
    exp = hist.sum() / 16
    assert ((hist - exp) ** 2 / exp).sum() < 37.7  # chi-square, 15 dof, p = 1e-3


def _ggx_albedo_quadrature(wo, alpha, f0):
    """Directional albedo  int f(wo, wi) cos(theta_i) dwi  of the GGX microfacet BRDF
    f = F D G / (4 |wo.n| |wi.n|) (Walter et al. 2007), by a midpoint rule in (theta, phi)."""
    nt, nphi = 1500, 1200
    th = (np.arange(nt) + 0.5) * (np.pi / 2) / nt
    ph = (np.arange(nphi) + 0.5) * (2 * np.pi) / nphi
    T, P = np.meshgrid(th, ph, indexing="ij")
    wi = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], axis=-1)
    h = wi + wo
    h /= np.linalg.norm(h, axis=-1, keepdims=True)
    ch = h[..., 2]
    a2 = alpha * alpha
    tan2h = (1 - ch ** 2) / ch ** 2
    D = a2 / (np.pi * ch ** 4 * (a2 + tan2h) ** 2)

    def G1(z):
        t2 = np.maximum(0, (1 - z ** 2) / z ** 2)
        return 2 / (1 + np.sqrt(1 + a2 * t2))

    G = G1(wo[2]) * G1(wi[..., 2])
    hd = (wi * h).sum(-1)
    out = []
    for f in f0:
        F = f + (1 - f) * (1 - hd) ** 5
        fr = F * D * G / (4 * wo[2] * wi[..., 2])
        integrand = fr * wi[..., 2] * np.sin(T)
        out.append(integrand.sum() * (np.pi / 2 / nt) * (2 * np.pi / nphi))
    return np.array(out)


@pytest.mark.parametrize("alpha", [0.15, 0.3, 0.5])
@pytest.mark.parametrize("theta_o_deg", [0.0, 35.0, 65.0])
def test_ggx_weight_matches_brdf_albedo(orc, alpha, theta_o_deg):
    """E[weight] of the sampler equals the albedo integral of the BRDF it claims to sample."""
    to = math.radians(theta_o_deg)
    wo = np.array([math.sin(to), 0.0, math.cos(to)])
    f0 = np.array([0.2, 0.5, 0.9])
    u1, u2 = _stratified(160)
    acc = np.zeros(3)
    for a, b in zip(u1, u2):
        ok, wi, wt = orc.sample_ggx(wo, alpha, f0, a, b)
        if ok:
            assert wi[2] > 0
            acc += wt
    mc = acc / u1.size
    ref = _ggx_albedo_quadrature(wo, alpha, f0)
    assert np.allclose(mc, ref, rtol=6e-3, atol=1e-3), (mc, ref)


def test_ggx_reflects_about_sampled_half_vector(orc):
    rng = np.random.default_rng(0)
    for _ in range(200):
        wo = rng.normal(size=3)
        wo[2] = abs(wo[2]) + 0.1
        wo = (wo / np.linalg.norm(wo)).astype(np.float32)
        ok, wi, wt = orc.sample_ggx(wo, 0.3, [0.5, 0.5, 0.5], rng.random(), rng.random())
        h = wi.astype(np.float64) + wo
        h /= np.linalg.norm(h)
        # law of reflection: equal angles to the half vector, unit length
        assert abs(np.dot(h, wo) - np.dot(h, wi)) < 1e-5
        assert abs(np.linalg.norm(wi) - 1) < 1e-5
        assert ok == (wi[2] > 0)


def test_frame_orthonormal(orc):
    rng = np.random.default_rng(1)
    ns = rng.normal(size=(2000, 3))
    ns = np.concatenate([ns, [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [0, 0, -1e-9]]])
    for n in ns:
        n = (n / np.linalg.norm(n)).astype(np.float32)
        t, b = orc.frame(n)
        M = np.stack([t, b, n]).astype(np.float64)
        assert np.abs(M @ M.T - np.eye(3)).max() < 5e-6
        assert np.allclose(np.cross(t, b), n, atol=5e-6)  # right-handed
