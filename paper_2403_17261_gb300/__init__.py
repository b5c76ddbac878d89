"""GB300 (sm_103a) implementation of the data-parallel hot path of Kale & Kry,
"Distributed Simulation of Large Multi-body Systems": every overlapping worker
is a partition solved by its own group of CTAs; overlap bodies are blended
with inverse-geodesic weights.

* ``ovl``         -- ctypes binding of libovl (C ABI in ``include/ovl.h``);
                     ``ovl.Simulation(scene)`` steps a scene on the GPU
* ``scenes``      -- seeded synthetic workloads (inputs only), including the
                     box workloads ``box_building`` and ``plank_bridge``
* ``learned``     -- the learned warm start: log, train, compare
* ``experiments`` -- the growth-depth / weights error protocol
* ``build``       -- nvcc build of ``_build/libovl.so``

A minimal run::

    from paper_2403_17261_gb300 import ovl, scenes
    sim = ovl.Simulation(scenes.pile_small())
    for _ in range(10):
        sim.step()
    state = sim.state()          # [n, 13]: position, quaternion, v, omega
"""
__all__ = ["ovl", "scenes", "learned", "experiments", "build"]
