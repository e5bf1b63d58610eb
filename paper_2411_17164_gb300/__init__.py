"""GB300-native X-MeshGraphNet message-passing hot path (arXiv 2411.17164).

Submodules are imported lazily so that ``paper_2411_17164_gb300.synth`` (the
seeded input generators) can be used without loading the CUDA library:

* ``synth``        -- seeded synthetic point clouds, targets and parameters
* ``xmgn``         -- ctypes binding of the C-ABI library ``libxmgn.so``: graph
                      building, partitioning, ``Model`` (forward, backward,
                      checkpoint offload, autotuner) and the
                      ``torch.autograd.Function`` wrapper ``XMGNLoss``
* ``build``        -- nvcc build of the library for sm_103a
* ``dist``         -- partition assignment to ranks and the rank-ordered
                      gradient sum
* ``profile_step`` -- a plain fwd+bwd driver for profilers
"""
