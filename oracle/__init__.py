"""FP64 CPU oracle for DIST differentiable sphere tracing (arXiv 1911.13225).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_1911_13225_b300``) never imports it and shares no code with it; the
only common dependency is ``synth`` (seeded weights, latents and cameras,
which hold none of the method's arithmetic).

Plain, slow, obviously correct numpy float64.  Every function cites the part
of the paper it follows:

* ``mlp``     -- DeepSDF decoder f(p, z) and its hand-derived chain rule
                 (Sec. 3.4 problem statement, Sec. B.1 architecture).
* ``camera``  -- pixel-centre rays and the depth formula (Sec. 3.3, Sec. A.4).
* ``tracer``  -- unit-sphere initialisation, aggressive sphere tracing,
                 convergence and outputs (Alg. 1, Sec. 3.2, Eq. 1, Sec. 3.3,
                 Sec. A.3), and coarse-to-fine tracing (Sec. 3.2).
* ``grad``    -- latent gradients: exact implicit form and the paper's
                 first-term approximation (Eq. 2, Sec. 3.4, Sec. B.2);
                 camera-extrinsic gradients of depth and silhouette
                 (Sec. 4.2, pose optimisation through the renderer).
* ``loss``    -- depth / normal / silhouette losses (Sec. 4.2.1, Eq. 4 of the
                 appendix, Sec. B.3).
* ``photo``   -- multi-view photometric loss: warp by the rendered depth,
                 bilinear sampling, visibility test, L1 (Sec. 4.2, Sec. B.3).
* ``sdf``     -- analytic SDFs used as pins (sphere, box, plane, slab).
* ``brute``   -- dense fixed-step first-root search used as a pin.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` except
the paper's approximated gradient (``grad.paper_depth_grad``), whose value as
an approximation of the true gradient has no reference to compare against:
parity unpinned (its arithmetic is pinned on an analytic SDF only); and
what a child ray inherits in coarse-to-fine tracing
(``tracer.render_coarse_to_fine``), which the paper does not state: parity
unpinned as a reading of the paper (the code is pinned against a scalar
restatement of the reading, an exact sphere and the plain tracer).
"""
