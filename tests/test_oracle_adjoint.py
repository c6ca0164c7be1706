"""Pins of the oracle's reverse mode against FP64 central finite differences of the
oracle's own forward stepper."""
import numpy as np
import pytest

from oracle import adjoint as ad
from oracle import stepper as st
from paper_2302_08694_gb300 import workloads as wl


def mesh_case():
    Xref, tri = wl.latlong_sphere(3, 6, 0.25, (0.5, 0.5, 0.5))
    X = 0.5 + (Xref - 0.5) * np.array([[1.15], [0.9], [1.05]])
    return Xref, tri, X


@pytest.mark.parametrize("sigma", [1.0, 0.7])
def test_velocity_vjp_matches_fd(sigma):
    Xref, tri, X = mesh_case()
    N, mu = 6, 1.0
    force = st.mesh_model(Xref, tri, sigma)
    rng = np.random.default_rng(0)
    lam = rng.standard_normal(X.shape)
    v = rng.standard_normal(X.shape)
    gX, gs = ad.stokes_velocity_vjp(X, lam, force, sigma, N, mu)
    eps = 1e-6
    Up = st.stokes_velocity(X + eps * v, force, N, mu)
    Um = st.stokes_velocity(X - eps * v, force, N, mu)
    fd = np.sum(lam * (Up - Um)) / (2 * eps)
    assert abs(fd - np.sum(gX * v)) <= 1e-6 * max(abs(fd), 1e-12) + 1e-10
    fp = st.stokes_velocity(X, st.mesh_model(Xref, tri, sigma + eps), N, mu)
    fm = st.stokes_velocity(X, st.mesh_model(Xref, tri, sigma - eps), N, mu)
    fds = np.sum(lam * (fp - fm)) / (2 * eps)
    assert abs(fds - gs) <= 1e-6 * abs(fds)


def test_rollout_gradient_matches_fd_3d():
    Xref, tri, X0 = mesh_case()
    N, mu, dt, K, sigma = 6, 1.0, 2e-3, 3, 1.0
    center, R = np.array([0.5, 0.5, 0.5]), 0.25
    force = st.mesh_model(Xref, tri, sigma)

    def loss_of(X0_, sig):
        f = st.mesh_model(Xref, tri, sig)
        X = X0_
        for _ in range(K):
            X = st.stokes_step(X, f, N, mu, dt)
        return ad.sphere_loss(X, center, R)[0]

    g0, gs, _ = ad.rollout_grad(X0, K, force, sigma, N, mu, dt, lambda X: ad.sphere_loss(X, center, R)[1])
    rng = np.random.default_rng(1)
    for _ in range(2):
        v = rng.standard_normal(X0.shape)
        eps = 1e-6
        fd = (loss_of(X0 + eps * v, sigma) - loss_of(X0 - eps * v, sigma)) / (2 * eps)
        assert abs(fd - np.sum(g0 * v)) <= 1e-6 * abs(fd)
    fds = (loss_of(X0, sigma + 1e-6) - loss_of(X0, sigma - 1e-6)) / 2e-6
    assert abs(fds - gs) <= 1e-6 * abs(fds)


def test_rollout_gradient_matches_fd_2d_curve():
    M, N, mu, dt, K = 24, 8, 1.0, 1e-3, 3
    X0 = wl.ellipse(M, 0.3, 0.2, (0.45, 0.55))
    sigma = 1.3
    center, R = np.array([0.45, 0.55]), 0.25
    force = st.curve_model(sigma)

    def loss_of(X0_):
        X = X0_
        for _ in range(K):
            X = st.stokes_step(X, force, N, mu, dt)
        return ad.sphere_loss(X, center, R)[0]

    g0, gs, _ = ad.rollout_grad(X0, K, force, sigma, N, mu, dt, lambda X: ad.sphere_loss(X, center, R)[1])
    v = np.random.default_rng(2).standard_normal(X0.shape)
    fd = (loss_of(X0 + 1e-6 * v) - loss_of(X0 - 1e-6 * v)) / 2e-6
    assert abs(fd - np.sum(g0 * v)) <= 1e-6 * abs(fd)
