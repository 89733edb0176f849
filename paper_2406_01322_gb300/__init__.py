"""GB300-native pseudo-spectral channel solver: Navier-Stokes (wall-normal velocity-vorticity form)
coupled with a Cahn-Hilliard phase field, Fourier x Fourier x Chebyshev-tau, one GPU.

The compute path is the C-ABI library ``libchflow.so`` built from ``csrc/`` (hand-written sm_103a
CUDA kernels).  ``paper_2406_01322_gb300.binding`` is the thin ctypes layer over it; importing this
package does not load the library, ``binding`` does, and it raises if the library is missing.
"""
__all__ = ["inputs", "binding"]
