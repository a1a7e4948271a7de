"""GB300-native aggregation-AMG preconditioned Krylov solver (arXiv 2007.00056).

``paper_2007_00056_gb300.amg`` is the Python binding of the C ABI declared in
``include/amg.h``; ``paper_2007_00056_gb300.workloads`` generates the seeded
synthetic systems.  The binding is imported on demand so that the generators
work on machines without a GPU.
"""

__all__ = ["amg", "workloads", "build"]


def __getattr__(name):
    if name in ("amg", "workloads", "build"):
        import importlib

        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
