"""Stated accuracy of the precision modes against the float64 path.

The mixed mode (float32 x/y transforms and products, float64 along z) differs from the float64
step by float32 rounding of the products and transforms.  The measure per field is
max |a - b| / max |b| over the unpadded grid after the large channel's 200 steps
(512 x 256 x 257, Re_tau = 300, 64 drops), starting from the same fields.  The rounding of the
products u_i u_j, of size max|u|^2, enters every velocity component with about the same absolute
size, so v and w, about 1000 times smaller than u in that flow, carry about 1000 times the
relative error of u; against the velocity scale max|u| ("velocity_scale", the largest of the
three components' max |a - b| / max |u|) all three stay below 1e-5.  mass, kinetic, grad2 and
free_energy are relative differences of the diagnostics (phi's mass is conserved by the scheme
only to the truncation of the mean line's tau rows, so float32 rounding of the mean products
moves it at the 1e-9 level).
"""

MIXED_BOUNDS = {"u": 1e-5, "v": 2e-3, "w": 2e-3, "phi": 5e-5, "velocity_scale": 1e-5,
                "mass": 1e-8, "kinetic": 1e-6, "grad2": 1e-6, "free_energy": 1e-6}
