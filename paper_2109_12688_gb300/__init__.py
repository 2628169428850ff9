"""GB300-native Nesterov-accelerated ADMM diffeomorphic registration.

The compute path is the C-ABI library ``libnadmm.so`` (hand-written sm_103a
CUDA) built in-tree by ``__graft_entry__.build()``; ``nadmm`` is its thin
ctypes binding.  ``synth`` generates seeded synthetic inputs.
"""
