"""Test-side helpers: staggered coordinates and analytic fields.  Plain
numpy; holds none of the method's arithmetic."""
import numpy as np


def node_coords(g, c):
    """(Z, Y, X) broadcastable coordinate arrays of component c's nodes
    (c = 0,1,2 for u,v,w; 3 for cell centres)."""
    nx, ny, nz = g.nx, g.ny, g.nz
    ox = 0.0 if c == 0 else 0.5
    oy = 0.0 if c == 1 else 0.5
    oz = 0.0 if c == 2 else 0.5
    nyc = ny + 1 if c == 1 else ny
    x = (np.arange(nx) + ox) * g.dx
    y = (np.arange(nyc) + oy) * g.dy
    z = (np.arange(nz) + oz) * g.dz
    return z[:, None, None], y[None, :, None], x[None, None, :]


def sample(g, c, fn):
    Z, Y, X = node_coords(g, c)
    return np.ascontiguousarray(np.broadcast_to(fn(X, Y, Z), (g.nz, (g.ny + 1 if c == 1 else g.ny), g.nx)),
                                dtype=np.float64)


def ddx(fn, axis, h=1e-6):
    """Central difference of an analytic function along axis 0/1/2 (x/y/z)."""
    def d(X, Y, Z):
        a = [X, Y, Z]
        ap = list(a); am = list(a)
        ap[axis] = a[axis] + h
        am[axis] = a[axis] - h
        return (fn(*ap) - fn(*am)) / (2 * h)
    return d


def order(e1, e2, ratio=2.0):
    return np.log(e1 / e2) / np.log(ratio)
