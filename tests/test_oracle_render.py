"""Pins of the oracle's interface image (oracle.render) against closed-form geometry: one
spherical drop of radius R seen from outside the box."""
import math

import numpy as np

from oracle import render
from oracle.channel import Channel, Params
from paper_2406_01322_gb300 import inputs

R = 0.5
P = dict(nx=32, ny=32, nz=33, lx=2.0, ly=2.0, re_tau=50.0, ch=0.1, pe=10.0, dt=1e-3)
EYE, TARGET, UP, FOV = (1.0, -3.0, 0.0), (1.0, 1.0, 0.0), (0.0, 0.0, 1.0), 30.0


def drop_channel():
    p = Params(**P)
    c = Channel(p)
    u, v, w, phi = inputs.initial_fields(p.nx, p.ny, p.nz, p.re_tau, p.ch, 1, R, 1, amp=0.0,
                                         lx=p.lx, ly=p.ly)
    z = np.zeros_like(phi)
    c.set_fields(z, z, z, phi)        # the drop at rest, centred at (1, 1, 0)
    return c


def test_drop_silhouette_depth_and_shading():
    W = H = 64
    rgb, depth = render.render(drop_channel(), W, H, EYE, TARGET, UP, FOV)
    d = render.camera_rays(W, H, EYE, TARGET, UP, FOV)
    e, c = np.array(EYE), np.array([1.0, 1.0, 0.0])
    # distance from the centre to each ray line; the analytic first hit of the sphere
    t_c = np.sum((c - e) * d, axis=-1)
    miss2 = np.sum((c - e) ** 2) - t_c ** 2
    inside = miss2 < R * R
    t_hit = t_c - np.sqrt(np.where(inside, R * R - miss2, 0.0))
    hits = depth >= 0
    # silhouette: only pixels on the rim may differ (interface width sqrt(2) Ch ~ 2 dx)
    assert np.sum(hits != inside) <= 0.06 * np.sum(inside)
    rim = np.abs(np.sqrt(miss2) - R) < 0.06
    assert np.all((hits == inside) | rim)
    # depth of the hits away from the rim: the zero level of the interpolated tanh profile
    core = hits & inside & (np.sqrt(miss2) < 0.8 * R)
    assert np.max(np.abs(depth[core] - t_hit[core])) < 0.01
    # shading: facing pixels are lit fully (|n . d| ~ 1), background elsewhere
    mid = rgb[H // 2, W // 2].astype(int)
    assert np.all(np.abs(mid - np.round(255 * render.DROP)) <= 3)
    assert tuple(rgb[0, 0]) == tuple(np.floor(255 * render.BACKGROUND + 0.5).astype(np.uint8))


def test_flat_interface_depth_is_exact():
    # phi = z - 0.2 is linear in z, so its interpolant is exact and the hit is exact up to the
    # bisection resolution (step / 2^40)
    p = Params(**P)
    c = Channel(p)
    X, Y, Z = np.meshgrid(np.arange(p.nx) * p.lx / p.nx, np.arange(p.ny) * p.ly / p.ny,
                          np.cos(np.pi * np.arange(p.nz) / (p.nz - 1)), indexing="xy")
    Z = np.transpose(Z, (2, 0, 1))
    zero = np.zeros_like(Z)
    c.set_fields(zero, zero, zero, Z - 0.2)
    eye, target = (1.0, 1.0, 3.0), (1.0, 1.0, 0.0)
    rgb, depth = render.render(c, 16, 16, eye, target, (0.0, 1.0, 0.0), 20.0)
    d = render.camera_rays(16, 16, eye, target, (0.0, 1.0, 0.0), 20.0)
    t_exact = (0.2 - eye[2]) / d[..., 2]
    assert np.max(np.abs(depth - t_exact)) < 1e-9
    # the gradient (0, 0, 1) against the ray: lambda = |d_z|
    lam = np.abs(d[..., 2])
    want = np.floor(255 * render.DROP[None, None, :] * (0.25 + 0.75 * lam)[..., None] + 0.5)
    assert np.max(np.abs(rgb.astype(int) - want)) <= 1
