"""Oracle for the learned proposal network (filled in with oracle/mlp.c)."""


def _register(L):
    return L
