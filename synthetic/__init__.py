from .scenes import *  # noqa
