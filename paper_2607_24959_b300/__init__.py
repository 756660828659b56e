"""B300-native batched regularised smooth-contact solve and its IFT adjoint.

The solve and its adjoint run in hand-written CUDA kernels for sm_103a behind
the C ABI in ``include/contact_solve.h`` (``libcs_b300.so``, built in-tree by
``paper_2607_24959_b300.build``).  Submodules:

* ``solver``    ``solve_fwd`` / ``solve_adjoint`` / ``solve_fused`` on torch tensors
* ``autograd``  ``ContactSolve`` torch.autograd.Function (IFT backward)
* ``workloads`` seeded synthetic inputs (no solver arithmetic)

Importing the package does not load the CUDA library; the first call does,
and it raises if the library is missing.
"""

__all__ = ["solver", "workloads", "build"]
