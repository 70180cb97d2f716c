"""FP64 CPU oracle for the R-MATEX integrator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The product (the CUDA library and its Python binding) never imports it, and
this package imports nothing from the product.  Both sides share only the
seeded input generator ``gridgen``.

Modules
-------
rmatex_ref   forward R-MATEX (Alg. 1 + Alg. 2 with the shift-and-invert
             specialisation of Sec. 3.3.2), the trapezoidal reference of
             Eq. 2, and the dense augmented-exponential reference of Eq. 4.
adjoint_ref  hand-written discrete reverse of rmatex_ref's forward pass.
"""
