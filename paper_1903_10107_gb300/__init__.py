"""GB300-native quantised LDPC reconciliation decoder (Mao et al., section 3).

Importing the package loads nothing; the CUDA library is built/loaded on the
first call that needs it (see :mod:`.native`)."""

__all__ = ["QCCode", "native", "inputs", "rate"]


def __getattr__(name):
    if name == "QCCode":
        from .decoder import QCCode
        return QCCode
    raise AttributeError(name)
