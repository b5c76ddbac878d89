"""GB300 (sm_103a) implementation of the data-parallel hot path of Kale & Kry,
"Distributed Simulation of Large Multi-body Systems": every overlapping worker
is a partition solved by its own CTA; overlap bodies are blended with
inverse-geodesic weights.

* ``ovl``    -- ctypes binding of libovl (C ABI in ``include/ovl.h``)
* ``scenes`` -- seeded synthetic workloads (inputs only)
* ``build``  -- nvcc build of ``_build/libovl.so``
"""
__all__ = ["ovl", "scenes", "build"]
