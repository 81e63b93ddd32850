"""GB300-native (sm_103a) fully algebraic H(curl) AMG: C-ABI library libamgh and its binding."""
from . import build  # noqa: F401
