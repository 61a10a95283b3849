"""FP64 CPU oracle for the 2D vesicle boundary-integral time step (VesNet, arXiv 2606.25569).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct restatement of
what the method computes, written from the paper's equations in double precision with numpy.
Only the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference legs of
``bench.py`` may import it. The CUDA library never calls it, shares no code with it, and
the product path fails loudly instead of falling back to it.

Modules, each citing the paper passage it follows:

* ``spectral``     -- Fourier derivative, arclength derivative, geometry (Sec. 2.2.1).
* ``stokes``       -- 2D Stokeslet (Eq. Stokeslet), self single layer with the Kress
                      log-singular product rule, trapezoid single layer (Sec. 2.2.2).
* ``operators``    -- B, T, P, L, M of Eqs. bending_op .. PTop.
* ``flows``        -- shear (Sec. 5.4), Poiseuille (Sec. 5.3), Taylor-Green (Eq. tayGreenFlow).
* ``farfield``     -- all-pairs far-field sum with the near-field mask (Sec. 2.2.2, 4.1).
* ``redistribute`` -- equal-arclength redistribution (Sec. 4.2).
* ``correct``      -- area/length correction as the exact constrained minimiser (Sec. 4.3).
* ``nearfield``    -- five layers + Gaussian RBF interpolation (Sec. 3.3, App. A).
* ``standardize``  -- centre / principal axis / reorder / unit length (Sec. 3.4.1).
* ``mlp``          -- FP64 MLP forward, backward, loss and AdamW (Sec. 3.4.2).
* ``step``         -- one plain time step in the order of Algorithm 1 with exact operators
                      (Eqs. advection_disc, relaxation_disc, tension_disc).

Parity-unpinned functions are listed in each module's header.
"""
