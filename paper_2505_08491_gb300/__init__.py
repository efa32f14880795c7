"""GB300 (sm_103a) library for the neural-preconditioned solve of the
discretised 3D-1D coupled elliptic problem (arXiv 2505.08491).

The compute path is the C-ABI shared library ``libmd_gb300.so`` (declared in
``include/md.h``); this package is its Python binding.  Importing the package
does not load the library; the first use does, and raises if it is missing.
"""
from .api import SMOOTH_OMEGA, Batch, Network, NetworkFunction, Operator, UNet, assemble, train, train_loss  # noqa: F401

__all__ = ["Operator", "assemble", "Network", "NetworkFunction", "UNet", "Batch", "train", "train_loss", "SMOOTH_OMEGA"]
