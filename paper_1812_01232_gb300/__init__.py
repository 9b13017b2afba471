"""GB300 (sm_103a) implementation of the GOSMA branch-and-bound hot path
(Campbell et al., "The Alignment of the Spheres: Globally-Optimal Spherical
Mixture Alignment for Camera Pose Estimation").

* ``gosma``  - binding of the C ABI library libgosma.so (include/gosma.h)
* ``synth``  - seeded synthetic workloads
* ``build``  - nvcc build of the library
"""
__all__ = ["gosma", "synth", "build"]
