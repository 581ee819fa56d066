"""Oracle: a plain, slow, FP64 CPU implementation of the nodal DG hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it.

What it computes (the paper's application, §5: MIRGE-Com's nodal DG for
compressible, multi-species, viscous flow, advanced by explicit RK4; DOFs local
to each element in an array layout, §1 Fig. 1).  The paper names these pieces
but writes out none of their formulas, so every function follows the textbook
nodal DG the paper cites for its setting (Hesthaven & Warburton 2007, cited in
§1) and the classical definitions it names:

* ``refelem``   reference tetrahedron: Vandermonde, Dr/Ds/Dt, mass, face mass,
                LIFT, Fmask (plain definitions: monomial basis, exact
                simplex integrals).
* ``geometry``  affine geometric factors, normals, face Jacobians; face
                connectivity of periodic meshes by coordinate matching.
* ``euler``     Euler fluxes, Lax-Friedrichs flux, strong- and weak-form DG
                right-hand sides (§5.2).
* ``ns``        compressible Navier-Stokes with BR1 gradients (§5.3).
* ``thermo``    perfect gas and NASA-7 mixture, Newton temperature solve and a
                bisection check (§4, §5: multi-species).
* ``lsrk``      Carpenter-Kennedy 5-stage 2N-storage RK4 and classical RK4 (§5.2).

Arrays follow the paper's layout: a field is [K][Np] (element, node), a state
is [V][K][Np].  Everything is float64.
"""
