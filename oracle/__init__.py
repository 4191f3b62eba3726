"""Plain FP64 CPU oracle for the collided-proton DLRA method of arXiv 2508.04484.

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it. The product library
(``paper_2508_04484_gb300``) never imports it, and it never imports the
product library: the two share no code.

Modules (each function cites the part of the paper it follows):

* ``angular``  -- real spherical harmonics, A_x/A_y/A_z and their eigen-split
                  (Sec. 3.3.1, Sec. 3.3.2).
* ``physics``  -- Bragg-Kleeman stopping power, scattering power, screened
                  Rutherford Legendre moments, extended transport correction
                  (Sec. 2.1, Sec. 2.1.1, Sec. 3.3.1).
* ``grid``     -- second-order one-sided stencils D^{+/-}_{x,y,z} (Sec. 3.3.2).
* ``problem``  -- per-energy coefficient evaluation for one configuration.
* ``raytrace`` -- CSDA uncollided ray tracer (Sec. 3.2, without straggling).
* ``fullrank`` -- full-rank solve with the same split and integrators (Sec. 4).
* ``dlra``     -- the augmented-BUG low-rank energy step (Sec. 2.2, Sec. 3.3.3).
* ``adjoint``  -- discrete adjoint of the full-rank solve: gradients of a loss of the
                  deposited energy with respect to beam and mixture weights.
* ``straggling`` -- uncollided energy distribution along a ray with straggling: energy
                  DG (P2, Lax-Friedrichs slowing down, SIPG straggling), Crank-Nicolson in
                  depth (Sec. 3.2); the GPU path does not have it yet.

Parity status of each function is stated in its module header; where a
function has no independent pin it says "parity unpinned".
"""
