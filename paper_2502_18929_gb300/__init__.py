"""GB300 (sm_103a) real-time population-dynamics QMC for noisy circuits
(Shen & Lidar, arXiv:2502.18929).

* ``qmc``      -- ctypes binding of the C ABI (include/qmc.h)
* ``problems`` -- master-equation descriptions and seeded synthetic inputs
* ``planner``  -- step-size planning at pulse-window boundaries
* ``build``    -- in-tree nvcc build of ``_lib/libqmc_gb300.so``
"""
