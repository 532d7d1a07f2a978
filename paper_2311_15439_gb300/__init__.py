"""GB300 (sm_103a) simplex-grid hash encoding (arXiv 2311.15439).

Submodules (imported on demand so that the seeded input generators in ``synth``
load without torch or the CUDA library):

* ``build``    -- compiles ``csrc/*.cu`` into ``libsimplexenc.so`` for sm_103a;
* ``_lib``     -- ctypes declarations of the C ABI (``include/simplexenc.h``);
* ``api``      -- ``Encoder``, ``Mlp``, ``Adam``: tensor-argument wrappers of the C ABI;
* ``autograd`` -- ``torch.autograd.Function`` wrappers;
* ``trainer``  -- the training step of the image / SDF workloads;
* ``serve``    -- continuous-batching query server for trained fields;
* ``synth``    -- seeded synthetic inputs.
"""
