"""Plain, slow FP64 CPU oracle for the F-Hash hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never calls
it, and the two share no code: the only common dependency is the ``synth``
package of seeded input generators, which holds none of the method's arithmetic.

Every routine follows the paper's definitions in its own notation and order:

* ``schedule``  - level resolutions: fold policy (Section 3.2.1 Eqs. 4-8, temporal
  policy of Section 3.2.2), plus explicit and geometric schedules; table sizes.
* ``index``     - feature dilation, per-frame bounding boxes, the Feature Bounding
  Box and the occupancy grid (Section 3.1).
* ``encode``    - the four encoding steps of Section 3.2.4: neighbouring time
  steps, embedding cell, 16 look-ups through the F-Hash of Eq. 9, quadrilinear
  interpolation of Eqs. 10-12; and the scatter of its backward pass.
* ``mlp``       - the shallow ReLU MLP, MSE loss and its analytic backward.
* ``adam``      - Adam as used for training (Section 5.1.3), PyTorch semantics.
* ``rng``       - SplitMix64 counter-based values used to check device-side init.
* ``render``    - sample-streaming renderer with adaptive ray marching (Algorithm 1,
  Section 3.3) and the time-slice decode.

Where the paper is silent or garbled the reading taken is stated beside the
code; the one FP32 step (cell location) is done
in float32 on purpose, because it decides integer table rows and both sides must
take that decision in the same precision.
"""
