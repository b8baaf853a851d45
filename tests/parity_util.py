"""Element-wise comparison of type-major vectors, one variable type at a time.

The five types of the lifted system (u, v, z, lambda, mu; Fig. 4) carry very
different scales in the scaled coordinates of Sec. 4.1 (mu is O(1/dt) larger
than lambda, z is weighted by gamma), so one 2-norm over the whole vector can
hide an error confined to one type.  These helpers bound the largest entry
error of each type by that type's largest reference entry.
"""
import numpy as np

TYPES = ("u", "v", "z", "lambda", "mu")


def type_slices(n, p, q):
    """Slices of u, v, z, lambda, mu in a type-major vector of n (4p + q) entries."""
    widths = (p, p, q, p, p)
    out, start = {}, 0
    for name, w in zip(TYPES, widths):
        out[name] = slice(start, start + n * w)
        start += n * w
    return out


def per_type_errors(x, ref, n, p, q):
    """{type: max|x - ref| / max|ref|} over the entries of each variable type."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    errs = {}
    for name, sl in type_slices(n, p, q).items():
        scale = float(np.max(np.abs(ref[sl]))) if ref[sl].size else 0.0
        diff = float(np.max(np.abs(x[sl] - ref[sl]))) if ref[sl].size else 0.0
        errs[name] = diff / scale if scale > 0 else diff
    return errs


def assert_per_type(x, ref, n, p, q, tol, what=""):
    errs = per_type_errors(x, ref, n, p, q)
    worst = max(errs, key=errs.get)
    assert errs[worst] <= tol, f"{what} {worst}: {errs[worst]:.3e} > {tol:.1e} ({errs})"
    return errs
