"""Training of the learned FGMRES preconditioner on (residual, error) pairs.

For A x = z started from x_0 = 0, the residual of the start is r = z and its
error is e = x* - x_0 = A^-1 z, so every solve of the library's own batched
solver yields a pair (r, e) with A e = r.  The network M (dtr.Net) is trained
on such pairs with Adam, entirely on the GPU through the library's
forward/backward/Adam kernels, and is then used as the right preconditioner
of the FGMRES solver (solver="fgmres_net").  Two losses:

  * residual loss (default): sum_j |A M r_j - r_j|^2 / |r_j|^2, the quantity
    right preconditioning makes small; the error e is not needed;
  * error loss: sum_j |M r_j - e_j|^2 / |e_j|^2.

The network is a translation-invariant stencil that does not see the gauge
links, so it can only learn the disorder-averaged propagator: it gains where
the links are close to unit (weak disorder) and the mass is small, and gains
nothing at strong disorder.

train() cycles a fixed pool of pairs; train_stream() draws a fresh batch of
pairs from new solves at every step, so the number of distinct pairs (20k for
the 16^3x32 workload) is limited by time, not by memory (one pair of 16^3x32
fields is 50 MB).
"""
import numpy as np


def make_pairs(gauge, m0, nrhs, seed, first_run, tol=1e-6):
    """nrhs independent Z4 right-hand sides (runs first_run, first_run + 1, ...)
    and their solutions: residual/error pairs of the start x_0 = 0."""
    import torch

    from . import dtr
    lat = gauge.lat
    z = torch.cat([dtr.gen_noise(lat, seed, first_run + k, 1, False, 0, 1) for k in range(nrhs)])
    e, st = dtr.solve_batch(gauge, m0, z, params=dtr.solve_params(tol=tol, solver="mixed_f32"))
    return z, e


def train(net, gauge, m0, steps=100, batch=8, lr=3e-4, seed=12345, pool=8, residual_loss=True, log_every=0):
    """Train on `pool` batches of independent pairs (cycled); returns the loss
    history (mean per-column loss per step).  residual_loss: minimise
    |A M r - r|^2 / |r|^2 (else the error loss |M r - e|^2 / |e|^2)."""
    batches = [make_pairs(gauge, m0, batch, seed, r * batch) for r in range(pool)]
    hist = []
    for s in range(steps):
        z, e = batches[s % pool]
        loss = net.train_step(z, e, lr=lr, step=True, gauge=gauge if residual_loss else None, m0=m0) / batch
        hist.append(loss)
        if log_every and s % log_every == 0:
            print("step %d loss %.4e" % (s, loss))
    return np.array(hist)


def train_stream(net, gauge, m0, pairs=20000, batch=16, lr=3e-4, seed=54321, residual_loss=True, solve_tol=1e-6):
    """Train on `pairs` distinct (residual, error) pairs, `batch` new ones per Adam
    step from the library's own solves (runs seed-indexed, never reused).
    Returns (loss history, seconds in solves, seconds in training steps)."""
    import time

    import torch
    hist, t_solve, t_train = [], 0.0, 0.0
    steps = (pairs + batch - 1) // batch
    for s in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        z, e = make_pairs(gauge, m0, batch, seed, s * batch, tol=solve_tol)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        hist.append(net.train_step(z, e, lr=lr, step=True, gauge=gauge if residual_loss else None, m0=m0) / batch)
        torch.cuda.synchronize()
        t_solve += t1 - t0
        t_train += time.perf_counter() - t1
    return np.array(hist), t_solve, t_train
