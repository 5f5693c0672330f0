"""Algorithm 1 (deflatedHP) and the statistics around it (oracle).

deflated_hp evaluates the estimator of Algorithm 1 (Section 5.2) in the order
the paper gives it: the deflated part T_D = Tr(Lambda^-1 V^H A^H V) once; then,
for each probing vector z = z0 .* z_h in turn (z0 and z_h drawn by
oracle.noise), the solution y of A y = z and the sample z^H y minus the
deflation term z^H V Lambda^-1 V^H (A^H z), accumulated so that after j samples
the estimate is T_D plus the mean of the first j samples.

Statistics: error bars by the delete-1 jackknife of the mean over independent
runs with different z0 (Section 6.2; delete-1 is the reading taken here), and
the sample variance.  Variances use the complex form E|t - E t|^2, the form
eq. (1.2) evaluates.
"""
import numpy as np

from . import deflation as _defl


def deflated_hp(AH, solve, Z, V=None, sigma=None, group=1):
    """Run Algorithm 1 over the columns of Z (already z0 .* z_h).

    AH: sparse or dense A^H; solve: callable Z -> A^-1 Z (columns);
    V, sigma: deflation space (None = no deflation, T_D = 0).
    group: with 12-fold spin-colour dilution each probing vector z is split
    into `group` = 12 diluted columns whose quadratures add up to one sample
    (Section 1, dilution); group = 1 otherwise.
    Returns dict with T_D, per-column zy (z^H y) and defl (deflation term),
    per-sample t (sum over the group of z^H y - defl) and trace (the running
    estimate T_D + mean of the first j samples, for each j).
    """
    ncol = Z.shape[1]
    assert ncol % group == 0
    s = ncol // group
    TD = _defl.T_D(AH, V, sigma) if V is not None else 0.0
    zy = np.zeros(ncol, dtype=np.complex128)
    dq = np.zeros(ncol, dtype=np.complex128)
    Y = solve(Z)
    for q in range(ncol):
        z = Z[:, q]
        zy[q] = np.vdot(z, Y[:, q])
        dq[q] = _defl.quadrature(AH, V, sigma, z) if V is not None else 0.0
    t = np.zeros(s, dtype=np.complex128)
    trace = np.zeros(s, dtype=np.complex128)
    TR = 0.0
    for j in range(s):
        t[j] = np.sum(zy[j * group:(j + 1) * group] - dq[j * group:(j + 1) * group])
        TR = TR + t[j]
        trace[j] = TR / (j + 1) + TD
    return {"T_D": TD, "zy": zy, "defl": dq, "t": t, "trace": trace, "Y": Y}


def sample_variance(x):
    """Unbiased complex-form sample variance sum |x - mean|^2 / (n - 1)."""
    x = np.asarray(x)
    return float(np.sum(np.abs(x - x.mean()) ** 2) / (len(x) - 1))


def jackknife_mean(x):
    """Delete-1 jackknife: (mean, variance of the mean) for samples x."""
    x = np.asarray(x)
    n = len(x)
    loo = (x.sum() - x) / (n - 1)
    var = (n - 1) / n * np.sum(np.abs(loo - loo.mean()) ** 2)
    return x.mean(), float(var)
