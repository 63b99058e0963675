"""GB300-native per-timestep hot path of paces (co-evolving subspaces, arXiv 2603.07341).

The compute path is the CUDA library ``libpaces`` (sm_103a) behind the C ABI
declared in ``include/paces.h``; ``paper_2603_07341_gb300.binding`` marshals
arguments to it.  Importing this package does not load the library, so the
seeded workload descriptions in ``workloads`` stay usable on machines without
a GPU; the binding raises if the library is missing.

Modules: ``binding`` (the Solver class and plain calls), ``autograd`` (the
trajectory as a torch.autograd.Function over J, g, omega and the site
energies), ``autotune`` (launch shapes by timing steps), ``analysis``
(absorption spectrum and RMSD from the records), ``workloads`` (seeded model
descriptions), ``build`` (nvcc for sm_103a, in tree).
"""

__all__ = ["binding", "workloads", "build", "autograd", "autotune", "analysis"]
