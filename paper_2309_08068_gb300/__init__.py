"""GB300-native (sm_103a) lattice-Boltzmann Maxwell solvers: the Mendoza-Munoz (MM) and modified
Hauser-Verhey (HV) time steps of arXiv 2309.08068, behind the C-ABI library ``liblbm.so``.

``Lattice`` (in ``lbm``) is the Python binding; ``workloads`` builds seeded inputs. Importing the
package does not load the CUDA library; creating a ``Lattice`` does, and raises if it is missing.
"""

__all__ = ["Lattice", "workloads"]


def __getattr__(name):
    if name == "Lattice":
        from .lbm import Lattice
        return Lattice
    raise AttributeError(name)
