"""FP64 CPU oracle for the compressible fast-Eulerian PISO step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, literal restatement
of the discrete method in numpy (FP64 throughout).  It exists so that the CUDA
path can be checked element by element.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  The product path (``paper_1404_0959_gb300``)
never imports it and shares no code with it.

Source of the method (Cerminara, Berselli, Esposti Ongaro, Salvetti,
"Direct numerical simulation of a compressible multiphase flow through the
fast Eulerian approach", arXiv:1404.0959):

* Sec. 2, first paragraph: PISO pressure-velocity coupling, fourth-order
  central interpolation, adaptive time step.
* Sec. 2, second paragraph and its two footnotes: Fourier closure
  (q = -k grad T) and barotropic closure (p proportional to rho^gamma).
* Sec. 2, second/third paragraphs: Equilibrium-Eulerian particle velocity as
  the first-order Stokes-number expansion; Marble's dusty gas as its zero-order
  version.
* Sec. 1: decaying homogeneous isotropic turbulence at r.m.s. Mach 0.2 / 0.5.

The paper prints no equations for any of these, so every discrete formula
here is this project's reading of those passages.  Modules:

``ops``     fourth-order face interpolation and the face/cell stencils
``ic``      SplitMix64 counter RNG, Box-Muller, spectral solenoidal field
``piso``    one PISO step (predictor, two correctors, closures, dust)
``krylov``  Jacobi-PCG, Jacobi-BiCGStab, flexible CG, flexible GMRES
``diag``    kinetic energy, enstrophy, Taylor microscale, spectrum, totals
``unet``    FP64 3D-conv U-Net forward/backward (learned preconditioner)
``les``     top-hat filter, Favre sub-grid stress, Smagorinsky model, a-priori statistics
``twofluid`` Eulerian two-fluid dust phase (own momentum, Stokes drag), after the gas step
``isosurface`` marching-tetrahedra iso-surface and orthographic z-buffer depth image

Parity status of each function is stated in its module header.
"""
