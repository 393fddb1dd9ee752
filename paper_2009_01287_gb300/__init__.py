"""GB300-native hp-DG subspace-correction solver.

The compute path is the C-ABI library built from `csrc/` (see `binding`);
`inputs` holds the seeded synthetic workloads.  Importing the package does not
load the library; `binding.lib()` does, and raises if it is missing.
"""
